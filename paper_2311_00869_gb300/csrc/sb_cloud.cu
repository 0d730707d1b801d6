// sb_cloud.cu -- the frustration cloud (Algorithm 1, Eq. 1): distinct
// balanced states with their count C and switch count S.
//
// The paper keys its std::map by the state's edge-sign string.  Here a state
// is its canonical vertex labelling (vertex 0 on the +1 side), which for a
// connected graph is in bijection with that string; the table is keyed by a
// 64-bit subset-sum hash of the labelling and every hash match is checked bit
// for bit against the stored state, so a hash collision never merges two
// states.  Stored states (the matrix B of the scalable variant) live in HBM
// chunk-major: bits[chunk][state], 64 vertices per word.
#include <algorithm>
#include <vector>

#include "sb_internal.cuh"

#define CL_DEFAULT_STATES 4096
#define CL_PARALLEL_ASSIGN 1  // one-block sorted assignment instead of the sequential pass

__host__ __device__ __forceinline__ uint64_t cl_slot_of(uint64_t key, int64_t slots)
{
    return (key ^ (key >> 29) ^ (key >> 47)) & (uint64_t)(slots - 1);
}

__host__ __device__ __forceinline__ uint64_t cl_key(uint64_t h, int bits)
{
    return bits >= 64 ? h : (h & ((1ull << bits) - 1ull));
}

// Sequential insertion in tree order (first appearance decides the state
// index).  One thread: the batch holds at most 4096 trees.
__global__ void k_cloud_assign(const uint64_t* __restrict__ hashes, const int32_t* __restrict__ counts, int64_t K,
                               int64_t tree_begin, int hash_bits, sb_cloud_slot* table, int64_t slots,
                               sb_cloud_entry* entries, int64_t max_states, int32_t* meta, int32_t* assign,
                               int32_t* rep, int32_t* mismatch)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t ns = meta[0];
    for (int64_t i = 0; i < K; i++) {
        const uint64_t h = hashes[i];
        const uint64_t key = cl_key(h, hash_bits);
        uint64_t s = cl_slot_of(key, slots);
        int32_t found = -1;
        int64_t probes = 0;
        while (table[s].state >= 0 && probes < slots) {
            if (table[s].key == key) {
                found = table[s].state;
                break;
            }
            s = (s + 1) & (uint64_t)(slots - 1);
            probes++;
        }
        mismatch[i] = 0;
        if (found >= 0) {
            entries[found].count += 1;
            assign[i] = found;
            if (entries[found].S != counts[i]) mismatch[i] = 1;  // certainly another state
        } else if (ns >= max_states || probes >= slots) {
            meta[1] += 1;
            assign[i] = -1;
        } else {
            table[s].key = key;
            table[s].state = ns;
            sb_cloud_entry e;
            e.hash = h;
            e.S = counts[i];
            e.count = 1;
            e.first_tree = tree_begin + i;
            entries[ns] = e;
            rep[ns] = (int32_t)i;
            assign[i] = ns;
            ns++;
        }
    }
    meta[0] = ns;
}

// The same assignment as k_cloud_assign, by one block: the batch's (key,
// tree) pairs are sorted, each run of one key is led by its smallest tree;
// leaders look their key up in the table; keys not found become new states,
// numbered in the order of their leaders' trees (what the sequential pass
// gives), and are inserted with atomicCAS on empty slots (no lookups run
// while they are inserted, and the keys are distinct).
#define CLP_THREADS 1024
__global__ void __launch_bounds__(CLP_THREADS)
    k_cloud_assign_par(const uint64_t* __restrict__ hashes, const int32_t* __restrict__ counts, int K,
                       int64_t tree_begin, int hash_bits, sb_cloud_slot* table, int64_t slots, sb_cloud_entry* entries,
                       int64_t max_states, int32_t* meta, int32_t* assign, int32_t* rep, int32_t* mismatch)
{
    extern __shared__ __align__(16) unsigned char clp_smem[];
    int P = 1;
    while (P < K) P <<= 1;
    uint64_t* key = (uint64_t*)clp_smem;       // P sorted keys
    int32_t* idx = (int32_t*)(key + P);        // P trees, sorted with the keys
    int32_t* runst = idx + P;                  // K: state of the run at each sorted position
    int32_t* isnew = runst + K;                // K, by tree: 1 for a leader of a new key; then its new index
    __shared__ int32_t s_part[CLP_THREADS / 32], s_ns, s_total;
    const int tid = threadIdx.x;
    const uint64_t mask = (uint64_t)(slots - 1);
    if (tid == 0) s_ns = meta[0];
    for (int i = tid; i < P; i += CLP_THREADS) {
        key[i] = i < K ? cl_key(hashes[i], hash_bits) : ~0ull;
        idx[i] = i < K ? i : 0x7FFFFFFF;
    }
    for (int i = tid; i < K; i += CLP_THREADS) isnew[i] = 0;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += CLP_THREADS) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[i] > key[p] || (key[i] == key[p] && idx[i] > idx[p]);
                    if (gt == up) {
                        const uint64_t tk = key[i];
                        key[i] = key[p];
                        key[p] = tk;
                        const int32_t ti = idx[i];
                        idx[i] = idx[p];
                        idx[p] = ti;
                    }
                }
            }
            __syncthreads();
        }
    // leaders look their key up; -2 marks a key to create
    for (int i = tid; i < K; i += CLP_THREADS) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        uint64_t s = cl_slot_of(key[i], slots);
        int32_t found = -1;
        for (int64_t p = 0; p < slots && table[s].state >= 0; p++) {
            if (table[s].key == key[i]) {
                found = table[s].state;
                break;
            }
            s = (s + 1) & mask;
        }
        runst[i] = found >= 0 ? found : -2;
        if (found < 0) isnew[idx[i]] = 1;
    }
    __syncthreads();
    // new indices in tree order: exclusive prefix of isnew over the trees
    {
        const int per = (K + CLP_THREADS - 1) / CLP_THREADS;
        const int b = tid * per, e = min(K, b + per);
        int32_t sum = 0;
        for (int t = b; t < e; t++) sum += isnew[t];
        int32_t inc = sum;
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if ((tid & 31) >= d) inc += y;
        }
        if ((tid & 31) == 31) s_part[tid >> 5] = inc;
        __syncthreads();
        if (tid < 32) {
            int32_t w = tid < CLP_THREADS / 32 ? s_part[tid] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (tid >= d) w += y;
            }
            if (tid < CLP_THREADS / 32) s_part[tid] = w;
            if (tid == 31) s_total = w;
        }
        __syncthreads();
        int32_t run = (tid >= 32 ? s_part[(tid >> 5) - 1] : 0) + inc - sum;
        for (int t = b; t < e; t++) {
            const int32_t f = isnew[t];
            isnew[t] = f ? s_ns + run : -1;  // the new state's index (may exceed capacity)
            run += f;
        }
    }
    __syncthreads();
    // leaders of new keys: create and insert (or overflow)
    for (int i = tid; i < K; i += CLP_THREADS) {
        if (runst[i] != -2) continue;
        const int32_t tl = idx[i];
        const int32_t st = isnew[tl];
        if (st >= max_states) {
            runst[i] = -1;
            continue;
        }
        uint64_t s = cl_slot_of(key[i], slots);
        for (int64_t p = 0; p < slots; p++) {
            if (atomicCAS(&table[s].state, -1, st) == -1) {
                table[s].key = key[i];
                break;
            }
            s = (s + 1) & mask;
        }
        sb_cloud_entry en;
        en.hash = hashes[tl];
        en.S = counts[tl];
        en.count = 0;
        en.first_tree = tree_begin + tl;
        entries[st] = en;
        rep[st] = tl;
        runst[i] = st;
    }
    __syncthreads();
    // every head hands its state to the rest of its run
    for (int i = tid; i < K; i += CLP_THREADS) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        for (int j = i + 1; j < K && key[j] == key[i]; j++) runst[j] = runst[i];
    }
    __syncthreads();
    // every tree: the state of its run, counts, overflow, S check
    for (int i = tid; i < K; i += CLP_THREADS) {
        const int32_t st = runst[i];
        const int32_t t = idx[i];
        assign[t] = st;
        mismatch[t] = 0;
        if (st < 0) {
            atomicAdd(&meta[1], 1);
            continue;
        }
        atomicAdd(&entries[st].count, 1);
        if (entries[st].S != counts[t]) mismatch[t] = 1;  // certainly another state
    }
    if (tid == 0) meta[0] = (int32_t)min((int64_t)s_ns + s_total, max_states);
}

// true when h lies in the cyclic interval (i, j] of a table of `slots` slots
__device__ __forceinline__ bool cl_in_cyc(uint64_t h, uint64_t i, uint64_t j)
{
    return i < j ? (h > i && h <= j) : (h > i || h <= j);
}

// Removes state st (key `key`) from the linear-probing table, moving later
// entries of the same run back (no tombstones).
__device__ void cl_table_erase(sb_cloud_slot* table, int64_t slots, uint64_t key, int32_t st)
{
    const uint64_t mask = (uint64_t)(slots - 1);
    uint64_t hole = cl_slot_of(key, slots);
    for (int64_t p = 0; p < slots && table[hole].state != st; p++) hole = (hole + 1) & mask;
    if (table[hole].state != st) return;
    uint64_t j = hole;
    for (int64_t p = 0; p < slots; p++) {
        j = (j + 1) & mask;
        if (table[j].state < 0) break;
        const uint64_t home = cl_slot_of(table[j].key, slots);
        if (!cl_in_cyc(home, hole, j)) {
            table[hole] = table[j];
            hole = j;
        }
    }
    table[hole].state = -1;
}

// The scalable rule (appendix algorithm alg-scale; the replaced state is one
// of largest S, the lowest such index): sequential in tree order.  The first
// stored state opens the cloud; later trees count only when their S is below
// the largest stored S; a new state is appended while fewer than fmax are
// stored, else it takes the slot of a largest-S state.  A replaced state that
// trees of this batch had matched loses those matches (assign = -1).
__global__ void k_cloud_assign_scalable(const uint64_t* __restrict__ hashes, const int32_t* __restrict__ counts,
                                        int64_t K, int64_t tree_begin, sb_cloud_slot* table, int64_t slots,
                                        sb_cloud_entry* entries, int64_t fmax, int32_t* meta, int32_t* assign,
                                        int32_t* rep, int32_t* touch, int32_t* mismatch)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t ns = meta[0];
    int32_t maxS = 0, arg = -1;
    auto rescan = [&]() {
        arg = -1;
        for (int32_t j = 0; j < ns; j++)
            if (arg < 0 || entries[j].S > maxS) {
                maxS = entries[j].S;
                arg = j;
            }
    };
    rescan();
    const uint64_t mask = (uint64_t)(slots - 1);
    for (int64_t i = 0; i < K; i++) {
        mismatch[i] = 0;
        assign[i] = -1;
        const uint64_t h = hashes[i];
        if (ns > 0 && !(counts[i] < maxS)) continue;
        uint64_t s = cl_slot_of(h, slots);
        int32_t found = -1;
        for (int64_t p = 0; p < slots && table[s].state >= 0; p++) {
            if (table[s].key == h) {
                found = table[s].state;
                break;
            }
            s = (s + 1) & mask;
        }
        if (found >= 0) {
            entries[found].count += 1;
            assign[i] = found;
            touch[found] = 1;
            if (entries[found].S != counts[i]) mismatch[i] = 1;  // certainly another state
            continue;
        }
        int32_t st;
        if (ns < fmax) {
            st = ns++;
        } else {
            st = arg;
            cl_table_erase(table, slots, entries[st].hash, st);
            if (touch[st])
                for (int64_t j = 0; j < i; j++)
                    if (assign[j] == st) {
                        assign[j] = -1;
                        mismatch[j] = 0;
                    }
            s = cl_slot_of(h, slots);  // the erase may have moved entries
            for (int64_t p = 0; p < slots && table[s].state >= 0; p++) s = (s + 1) & mask;
        }
        table[s].key = h;
        table[s].state = st;
        sb_cloud_entry e;
        e.hash = h;
        e.S = counts[i];
        e.count = 1;
        e.first_tree = tree_begin + i;
        entries[st] = e;
        rep[st] = (int32_t)i;
        touch[st] = 1;
        assign[i] = st;
        if (st == arg || ns == 1) rescan();  // a replacement, or the first state
    }
    meta[0] = ns;
}

// Canonical label bit of batch tree i at vertex v.
__device__ __forceinline__ uint32_t cl_bit(const uint64_t* row, const uint64_t* flipw, int64_t i)
{
    const int w = (int)(i >> 6), b = (int)(i & 63);
    return (uint32_t)(((row[w] ^ flipw[w]) >> b) & 1ull);
}

// One block per 64-vertex chunk.  For each tree of the batch: store the state
// (trees that created a state in this batch), or compare with the state it
// was matched to (its creator's labels, or the stored bits of an older state).
// The chunk's 64 label rows are staged in shared memory and turned into the
// trees' 64-vertex columns in place: a warp takes one word at a time and
// transposes its 64 x 64 bit block with four 32 x 32 warp transposes, so
// that slot [r][w] then holds the canonical column of tree 64 w + r.
#define CLV_THREADS 256
__global__ void __launch_bounds__(CLV_THREADS)
    k_cloud_verify(const uint64_t* __restrict__ lab, int64_t n, int W, const uint64_t* __restrict__ flipw, int64_t K,
                   const int32_t* __restrict__ assign, const int32_t* __restrict__ rep, uint64_t* bits,
                   int64_t max_states, int32_t* mismatch)
{
    extern __shared__ uint64_t rows[];  // 64 x W
    const int64_t chunk = blockIdx.x;
    const int64_t v0 = chunk * 64;
    const int nv = (int)min((int64_t)64, n - v0);
    for (int i = threadIdx.x; i < 64 * W; i += CLV_THREADS) {
        const int r = i / W, w = i - r * W;
        rows[i] = r < nv ? lab[(v0 + r) * W + w] : 0;
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t valid = nv >= 64 ? ~0ull : ((1ull << nv) - 1ull);
    for (int w = (int)(threadIdx.x >> 5); w < W; w += CLV_THREADS / 32) {
        const uint64_t a = rows[lane * W + w], b = rows[(lane + 32) * W + w];  // vertices lane, lane + 32
        const uint64_t lo = (uint64_t)warp_transpose32((uint32_t)a, lane) |
                            ((uint64_t)warp_transpose32((uint32_t)b, lane) << 32);          // tree 64 w + lane
        const uint64_t hi = (uint64_t)warp_transpose32((uint32_t)(a >> 32), lane) |
                            ((uint64_t)warp_transpose32((uint32_t)(b >> 32), lane) << 32);  // tree 64 w + 32 + lane
        const uint64_t f = flipw[w];
        rows[lane * W + w] = lo ^ (((f >> lane) & 1ull) ? valid : 0ull);
        rows[(lane + 32) * W + w] = hi ^ (((f >> (32 + lane)) & 1ull) ? valid : 0ull);
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < K; i += CLV_THREADS) {
        const int32_t s = assign[i];
        if (s < 0) continue;
        const uint64_t col = rows[(i & 63) * W + (i >> 6)];
        const int32_t creator = rep[s];
        uint64_t* slot = bits + chunk * max_states + s;
        if (creator == (int32_t)i) {
            *slot = col;
        } else {
            const uint64_t other = creator >= 0 ? rows[(creator & 63) * W + (creator >> 6)] : *slot;
            if (other != col) mismatch[i] = 1;
        }
    }
}

// Exact comparison (mode 0) or storage (mode 1) of one tree against one state.
__global__ void k_cloud_pair(const uint64_t* __restrict__ lab, int64_t n, int W, const uint64_t* __restrict__ flipw,
                             int64_t tree, int32_t state, uint64_t* bits, int64_t max_states, int mode, int32_t* differ)
{
    const int64_t nchunks = sb_cdiv(n, 64);
    for (int64_t chunk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; chunk < nchunks;
         chunk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = chunk * 64;
        const int nv = (int)min((int64_t)64, n - v0);
        uint64_t col = 0;
        for (int r = 0; r < nv; r++) col |= (uint64_t)cl_bit(lab + (v0 + r) * W, flipw, tree) << r;
        uint64_t* slot = bits + chunk * max_states + state;
        if (mode == 1) *slot = col;
        else if (*slot != col) atomicOr(differ, 1);
    }
}

__global__ void k_cloud_count(const int32_t* __restrict__ mismatch, int64_t K, int32_t* meta)
{
    int32_t c = 0;
    for (int64_t i = threadIdx.x; i < K; i += blockDim.x) c += mismatch[i];
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    __shared__ int32_t part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (unsigned i = 0; i < blockDim.x / 32; i++) t += part[i];
        meta[2] = t;
    }
}

__global__ void k_cloud_gather(const uint64_t* __restrict__ bits, int64_t nchunks, int64_t max_states, int64_t s,
                               uint64_t* out)
{
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += (int64_t)gridDim.x * blockDim.x)
        out[ch] = bits[ch * max_states + s];
}

sb_status sb_cloud_alloc(sb_ctx* c)
{
    if (c->cl_table) return SB_OK;
    if (c->cl_max <= 0) c->cl_max = CL_DEFAULT_STATES;
    if (c->cl_hash_bits <= 0 || c->cl_hash_bits > 64) c->cl_hash_bits = 64;
    int64_t slots = 1;
    while (slots < 2 * c->cl_max) slots <<= 1;
    c->cl_slots = slots;
    const int64_t nchunks = sb_cdiv(c->n, 64);
    c->cl_table = (sb_cloud_slot*)sb_dalloc(c, sizeof(sb_cloud_slot) * (size_t)slots);
    c->cl_entries = (sb_cloud_entry*)sb_dalloc(c, sizeof(sb_cloud_entry) * (size_t)c->cl_max);
    c->cl_bits = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)nchunks * (size_t)c->cl_max);
    c->cl_meta = (int32_t*)sb_dalloc(c, sizeof(int32_t) * 8);
    c->cl_assign = (int32_t*)sb_dalloc(c, sizeof(int32_t) * SB_TREES_MAX);
    c->cl_rep = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)c->cl_max);
    c->cl_mismatch = (int32_t*)sb_dalloc(c, sizeof(int32_t) * SB_TREES_MAX);
    c->cl_touch = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)c->cl_max);
    if (!c->cl_table || !c->cl_entries || !c->cl_bits || !c->cl_meta || !c->cl_assign || !c->cl_rep ||
        !c->cl_mismatch || !c->cl_touch) {
        sb_release_cloud(c);
        return sb_fail(c, SB_ERR_OOM, "cloud storage (%lld states)", (long long)c->cl_max);
    }
    // empty slots: state = -1 (all bytes 0xFF)
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->cl_table, 0xFF, sizeof(sb_cloud_slot) * (size_t)slots, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->cl_meta, 0, sizeof(int32_t) * 8, c->stream));
    c->cl_n_host = 0;
    return SB_OK;
}

// Rare path: trees whose hash matched a different state.  Each is re-probed
// on the host with an exact device comparison against every state sharing
// its key, and gets a new state when none is equal.
static sb_status cloud_resolve_collisions(sb_ctx* c)
{
    const int64_t K = c->K;
    std::vector<int32_t> assign(K), mism(K);
    std::vector<sb_cloud_slot> table(c->cl_slots);
    int32_t meta[8];
    SB_CHECK_CUDA(c, cudaMemcpyAsync(assign.data(), c->cl_assign, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(mism.data(), c->cl_mismatch, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(table.data(), c->cl_table, sizeof(sb_cloud_slot) * c->cl_slots,
                                     cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(meta, c->cl_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<sb_cloud_entry> entries(meta[0] + K);
    SB_CHECK_CUDA(c, cudaMemcpy(entries.data(), c->cl_entries, sizeof(sb_cloud_entry) * meta[0], cudaMemcpyDeviceToHost));
    std::vector<uint64_t> hashes(K);
    std::vector<int32_t> counts(K);
    SB_CHECK_CUDA(c, cudaMemcpy(hashes.data(), c->hashes, sizeof(uint64_t) * K, cudaMemcpyDeviceToHost));
    SB_CHECK_CUDA(c, cudaMemcpy(counts.data(), c->counts, sizeof(int32_t) * K, cudaMemcpyDeviceToHost));
    int32_t* differ = c->cl_meta + 4;
    int32_t ns = meta[0];
    const int64_t nchunks = sb_cdiv(c->n, 64);
    unsigned g = (unsigned)std::min<int64_t>(sb_cdiv(nchunks, 256), (int64_t)c->num_sms * 8);
    for (int64_t i = 0; i < K; i++) {
        if (!mism[i]) continue;
        entries[assign[i]].count -= 1;
        const uint64_t key = cl_key(hashes[i], c->cl_hash_bits);
        uint64_t s = cl_slot_of(key, c->cl_slots);
        int32_t found = -1;
        int64_t probes = 0;
        while (table[s].state >= 0 && probes < c->cl_slots) {
            if (table[s].key == key) {
                int32_t st = table[s].state;
                if (entries[st].S == counts[i]) {
                    int32_t h_differ = 0;
                    SB_CHECK_CUDA(c, cudaMemsetAsync(differ, 0, sizeof(int32_t), c->stream));
                    k_cloud_pair<<<g, 256, 0, c->stream>>>(c->labels, c->n, c->W, c->flipw, i, st, c->cl_bits,
                                                          c->cl_max, 0, differ);
                    SB_TRY(sb_after_launch(c, "k_cloud_pair"));
                    SB_CHECK_CUDA(c, cudaMemcpyAsync(&h_differ, differ, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                                     c->stream));
                    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
                    if (!h_differ) {
                        found = st;
                        break;
                    }
                }
            }
            s = (s + 1) & (uint64_t)(c->cl_slots - 1);
            probes++;
        }
        if (found >= 0) {
            entries[found].count += 1;
        } else if (ns >= c->cl_max || probes >= c->cl_slots) {
            meta[1] += 1;
        } else {
            table[s].key = key;
            table[s].state = ns;
            entries[ns].hash = hashes[i];
            entries[ns].S = counts[i];
            entries[ns].count = 1;
            entries[ns].first_tree = c->tree_begin + i;
            k_cloud_pair<<<g, 256, 0, c->stream>>>(c->labels, c->n, c->W, c->flipw, i, ns, c->cl_bits, c->cl_max, 1,
                                                  differ);
            SB_TRY(sb_after_launch(c, "k_cloud_pair"));
            ns++;
        }
    }
    meta[0] = ns;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(c->cl_table, table.data(), sizeof(sb_cloud_slot) * c->cl_slots,
                                     cudaMemcpyHostToDevice, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(c->cl_entries, entries.data(), sizeof(sb_cloud_entry) * ns, cudaMemcpyHostToDevice,
                                     c->stream));
    meta[2] = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(c->cl_meta, meta, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    return SB_OK;
}

sb_status sb_cloud_insert_batch(sb_ctx* c)
{
    if (c->batch_in_cloud) return SB_OK;
    SB_TRY(sb_cloud_alloc(c));
    SB_TRY(sb_score_batch(c));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->cl_rep, 0xFF, sizeof(int32_t) * (size_t)c->cl_max, c->stream));
    SbProf prof(c, SB_PROF_CLOUD);
    if (c->cl_fmax > 0) {
        SB_CHECK_CUDA(c, cudaMemsetAsync(c->cl_touch, 0, sizeof(int32_t) * (size_t)c->cl_max, c->stream));
        k_cloud_assign_scalable<<<1, 32, 0, c->stream>>>(c->hashes, c->counts, c->K, c->tree_begin, c->cl_table,
                                                         c->cl_slots, c->cl_entries, c->cl_fmax, c->cl_meta,
                                                         c->cl_assign, c->cl_rep, c->cl_touch, c->cl_mismatch);
        SB_TRY(sb_after_launch(c, "k_cloud_assign_scalable"));
    } else if (CL_PARALLEL_ASSIGN) {
        int P = 1;
        while (P < c->K) P <<= 1;
        const size_t smem = (sizeof(uint64_t) + sizeof(int32_t)) * (size_t)P + 2 * sizeof(int32_t) * (size_t)c->K;
        SB_CHECK_CUDA(c, cudaFuncSetAttribute(k_cloud_assign_par, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        k_cloud_assign_par<<<1, CLP_THREADS, smem, c->stream>>>(c->hashes, c->counts, (int)c->K, c->tree_begin,
                                                                c->cl_hash_bits, c->cl_table, c->cl_slots,
                                                                c->cl_entries, c->cl_max, c->cl_meta, c->cl_assign,
                                                                c->cl_rep, c->cl_mismatch);
        SB_TRY(sb_after_launch(c, "k_cloud_assign_par"));
    } else {
        k_cloud_assign<<<1, 32, 0, c->stream>>>(c->hashes, c->counts, c->K, c->tree_begin, c->cl_hash_bits,
                                                c->cl_table, c->cl_slots, c->cl_entries, c->cl_max, c->cl_meta,
                                                c->cl_assign, c->cl_rep, c->cl_mismatch);
        SB_TRY(sb_after_launch(c, "k_cloud_assign"));
    }
    const int64_t nchunks = sb_cdiv(c->n, 64);
    size_t smem = sizeof(uint64_t) * 64 * (size_t)c->W;
    if (smem > 48 * 1024)
        SB_CHECK_CUDA(c, cudaFuncSetAttribute(k_cloud_verify, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cloud_verify<<<(unsigned)nchunks, CLV_THREADS, smem, c->stream>>>(c->labels, c->n, c->W, c->flipw, c->K,
                                                                         c->cl_assign, c->cl_rep, c->cl_bits,
                                                                         c->cl_max, c->cl_mismatch);
    SB_TRY(sb_after_launch(c, "k_cloud_verify"));
    k_cloud_count<<<1, 1024, 0, c->stream>>>(c->cl_mismatch, c->K, c->cl_meta);
    SB_TRY(sb_after_launch(c, "k_cloud_count"));
    int32_t meta[4];
    SB_CHECK_CUDA(c, cudaMemcpyAsync(meta, c->cl_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (meta[2] > 0) {
        // a 64-bit hash shared by two different states: resolved exactly by the
        // unbounded cloud; the scalable one reports it instead
        if (c->cl_fmax > 0) return sb_fail(c, SB_ERR_DEVICE_CHECK, "state hash collision in the scalable cloud");
        SB_TRY(cloud_resolve_collisions(c));
    }
    c->batch_in_cloud = true;
    return SB_OK;
}

extern "C" sb_status sb_cloud_reset(sb_ctx* c, int64_t max_states, int32_t hash_bits)
{
    if (!c || max_states < 0 || max_states > (1ll << 30) || hash_bits < 0 || hash_bits > 64) return SB_ERR_ARG;
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    sb_release_cloud(c);
    c->cl_max = max_states > 0 ? max_states : CL_DEFAULT_STATES;
    c->cl_hash_bits = hash_bits > 0 ? hash_bits : 64;
    c->cl_fmax = 0;
    c->batch_in_cloud = true;  // a reset starts from the next sampled batch
    if (c->has_graph) SB_TRY(sb_cloud_alloc(c));
    return SB_OK;
}

extern "C" sb_status sb_cloud_reset_scalable(sb_ctx* c, int64_t f_max)
{
    if (!c || f_max < 1 || f_max > (1ll << 30)) return SB_ERR_ARG;
    SB_TRY(sb_cloud_reset(c, f_max, 64));
    c->cl_fmax = f_max;
    return SB_OK;
}

extern "C" sb_status sb_cloud(sb_ctx* c, sb_cloud_entry* out, int64_t cap, int64_t* n_states_out, int32_t* fr_min_out)
{
    if (!c || cap < 0 || (cap > 0 && !out) || !n_states_out) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_cloud_alloc(c));
    if (c->has_batch && !c->batch_in_cloud) SB_TRY(sb_cloud_insert_batch(c));
    int32_t meta[4];
    SB_CHECK_CUDA(c, cudaMemcpyAsync(meta, c->cl_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t ns = meta[0];
    c->cl_n_host = ns;
    *n_states_out = ns;
    const bool full = meta[1] > 0;
    if (!out && !fr_min_out)  // insertion only
        return full ? sb_fail(c, SB_ERR_CLOUD_FULL, "cloud capacity %lld reached; %d trees not stored",
                              (long long)c->cl_max, meta[1])
                    : SB_OK;
    std::vector<sb_cloud_entry> host(ns > 0 ? ns : 1);
    if (ns > 0)
        SB_CHECK_CUDA(c, cudaMemcpy(host.data(), c->cl_entries, sizeof(sb_cloud_entry) * ns, cudaMemcpyDeviceToHost));
    // order of first appearance (states created on the collision path are
    // numbered after the states of later trees of their batch)
    c->cl_order.resize(ns);
    for (int64_t i = 0; i < ns; i++) c->cl_order[i] = (int32_t)i;
    std::stable_sort(c->cl_order.begin(), c->cl_order.end(),
                     [&](int32_t a, int32_t b) { return host[a].first_tree < host[b].first_tree; });
    if (fr_min_out) {
        int32_t mn = -1;
        for (int64_t i = 0; i < ns; i++)
            if (mn < 0 || host[i].S < mn) mn = host[i].S;
        *fr_min_out = mn;
    }
    const int64_t k = std::min(ns, cap);
    if (k > 0) {
        std::vector<sb_cloud_entry> sorted(k);
        for (int64_t i = 0; i < k; i++) sorted[i] = host[c->cl_order[i]];
        SB_CHECK_CUDA(c, cudaMemcpy(out, sorted.data(), sizeof(sb_cloud_entry) * k, cudaMemcpyDefault));
    }
    if (full)
        return sb_fail(c, SB_ERR_CLOUD_FULL, "cloud capacity %lld reached; %d trees not stored", (long long)c->cl_max,
                       meta[1]);
    if (cap < ns && (cap > 0 || out))
        return sb_fail(c, SB_ERR_CLOUD_FULL, "output capacity %lld < %lld states", (long long)cap, (long long)ns);
    return SB_OK;
}

static sb_status cuda_st(sb_ctx* c, cudaError_t e, const char* what)
{
    return e == cudaSuccess ? SB_OK : sb_cuda_fail(c, e, what);
}

// Device copy of the canonical labels of cloud state `idx` (order of
// sb_cloud) in a buffer from sb_dalloc that the caller frees.
static sb_status cloud_state_dev(sb_ctx* c, int64_t idx, uint64_t** out)
{
    *out = nullptr;
    if (!c->has_graph || !c->cl_table) return sb_fail(c, SB_ERR_STATE, "no cloud");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    if (c->has_batch && !c->batch_in_cloud) SB_TRY(sb_cloud_insert_batch(c));
    int32_t ns = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&ns, c->cl_meta, sizeof(ns), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (idx < 0 || idx >= ns) return sb_fail(c, SB_ERR_ARG, "state index %lld out of [0, %d)", (long long)idx, ns);
    if ((int64_t)c->cl_order.size() != ns) {
        std::vector<sb_cloud_entry> host(ns);
        SB_CHECK_CUDA(c, cudaMemcpy(host.data(), c->cl_entries, sizeof(sb_cloud_entry) * ns, cudaMemcpyDeviceToHost));
        c->cl_order.resize(ns);
        for (int64_t i = 0; i < ns; i++) c->cl_order[i] = (int32_t)i;
        std::stable_sort(c->cl_order.begin(), c->cl_order.end(),
                         [&](int32_t a, int32_t b) { return host[a].first_tree < host[b].first_tree; });
    }
    idx = c->cl_order[idx];
    const int64_t nchunks = sb_cdiv(c->n, 64);
    uint64_t* tmp = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)nchunks);
    if (!tmp) return sb_fail(c, SB_ERR_OOM, "state export");
    k_cloud_gather<<<(unsigned)std::min<int64_t>(sb_cdiv(nchunks, 256), 4096), 256, 0, c->stream>>>(
        c->cl_bits, nchunks, c->cl_max, idx, tmp);
    sb_status st = sb_after_launch(c, "k_cloud_gather");
    if (st != SB_OK) {
        cudaStreamSynchronize(c->stream);
        sb_dfree(c, tmp);
        return st;
    }
    *out = tmp;
    return SB_OK;
}

extern "C" sb_status sb_cloud_state(sb_ctx* c, int64_t idx, uint64_t* bits_out)
{
    if (!c || !bits_out) return SB_ERR_ARG;
    uint64_t* tmp = nullptr;
    SB_TRY(cloud_state_dev(c, idx, &tmp));
    sb_status st = sb_copy_out(c, bits_out, tmp, sizeof(uint64_t) * (size_t)sb_cdiv(c->n, 64));
    cudaStreamSynchronize(c->stream);
    sb_dfree(c, tmp);
    return st;
}

// Edges whose sign the state switches: bit e of word e / 64 = lab[u] ^ lab[v]
// ^ neg of edge e (sb_graph_edges order).  One warp per 64-edge word.
__global__ void k_switch_edges(const int2* __restrict__ edges, int64_t m, const uint64_t* __restrict__ state,
                               uint64_t* __restrict__ out, unsigned long long* __restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t words = sb_cdiv(m, 64);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        uint32_t half[2];
        for (int h = 0; h < 2; h++) {
            const int64_t e = 64 * w + 32 * h + lane;
            uint32_t bit = 0;
            if (e < m) {
                const int2 ed = edges[e];
                const uint32_t u = (uint32_t)ed.x, v = (uint32_t)ed.y & SB_ID_MASK;
                bit = (uint32_t)(((state[u >> 6] >> (u & 63)) ^ (state[v >> 6] >> (v & 63))) & 1ull) ^
                      (ed.y < 0 ? 1u : 0u);
            }
            half[h] = __ballot_sync(0xffffffffu, bit);
        }
        if (lane == 0) {
            out[w] = ((uint64_t)half[1] << 32) | half[0];
            atomicAdd(count, (unsigned long long)(__popc(half[0]) + __popc(half[1])));
        }
    }
}

extern "C" sb_status sb_cloud_switch(sb_ctx* c, int64_t idx, uint64_t* edge_bits_out, int64_t* n_switched_out)
{
    if (!c || !edge_bits_out) return SB_ERR_ARG;
    uint64_t* state = nullptr;
    SB_TRY(cloud_state_dev(c, idx, &state));
    const int64_t words = sb_cdiv(c->m, 64);
    uint64_t* bits = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)std::max<int64_t>(words, 1));
    unsigned long long* cnt = (unsigned long long*)sb_dalloc(c, sizeof(unsigned long long));
    sb_status st = (bits && cnt) ? SB_OK : sb_fail(c, SB_ERR_OOM, "switch export");
    if (st == SB_OK) st = cuda_st(c, cudaMemsetAsync(cnt, 0, sizeof(*cnt), c->stream), "memset");
    if (st == SB_OK && words > 0) {
        const unsigned blocks = (unsigned)std::min<int64_t>(sb_cdiv(words * 32, 256), (int64_t)c->num_sms * 8);
        k_switch_edges<<<blocks, 256, 0, c->stream>>>(c->edges, c->m, state, bits, cnt);
        st = sb_after_launch(c, "k_switch_edges");
    }
    if (st == SB_OK) st = sb_copy_out(c, edge_bits_out, bits, sizeof(uint64_t) * (size_t)words);
    unsigned long long h = 0;
    if (st == SB_OK) st = cuda_st(c, cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
                                         "count copy");
    cudaStreamSynchronize(c->stream);
    if (st == SB_OK && n_switched_out) *n_switched_out = (int64_t)h;
    sb_dfree(c, state);
    sb_dfree(c, bits);
    sb_dfree(c, cnt);
    return st;
}

// ------------------------------------------------------ clouds of a batch
// One block per graph of a batch: the K trees of the graph are sorted by
// (hash, tree); every tree whose hash equals its run leader's is compared with
// the leader bit for bit over the graph's vertices, and a tree that differs
// starts its own state (matched, if possible, against the earlier differing
// trees of the run).  Output per graph: number of states, min S, and the
// states in order of first appearance.
#define BC_MAXK 1024
#define BC_THREADS 256

__device__ __forceinline__ uint32_t bc_bit(const uint64_t* lab, int W, const uint64_t* flip, int64_t v, int t)
{
    const int w = t >> 6;
    return (uint32_t)(((lab[v * W + w] ^ flip[w]) >> (t & 63)) & 1ull);
}

// 1 when trees a and b of the graph have equal canonical labels (whole warp)
__device__ bool bc_same(const uint64_t* lab, int W, const uint64_t* flip, int64_t v0, int64_t v1, int a, int b)
{
    uint32_t diff = 0;
    for (int64_t v = v0 + (threadIdx.x & 31); v < v1; v += 32) diff |= bc_bit(lab, W, flip, v, a) ^ bc_bit(lab, W, flip, v, b);
    return __all_sync(0xffffffffu, diff == 0);
}

__global__ void __launch_bounds__(BC_THREADS)
    k_batch_cloud(const uint64_t* __restrict__ hashes, const int32_t* __restrict__ counts, int64_t KP, int K,
                  const int64_t* __restrict__ tree0p, const uint64_t* __restrict__ lab, int W,
                  const uint64_t* __restrict__ flipw,
                  const int32_t* __restrict__ voff, int32_t* __restrict__ nstates_out, int32_t* __restrict__ frmin_out,
                  sb_cloud_entry* __restrict__ entries)
{
    __shared__ uint64_t key[BC_MAXK];
    __shared__ int32_t idx[BC_MAXK];
    __shared__ int32_t lead[BC_MAXK];   // sorted position -> position of its run leader
    __shared__ int32_t state[BC_MAXK];  // tree -> tree that represents its state
    __shared__ int32_t cnt[BC_MAXK];    // representative tree -> trees in its state
    __shared__ int32_t rank[BC_MAXK];   // representative tree -> output position
    __shared__ int32_t s_min, s_ns;
    const int64_t g = blockIdx.x;
    const uint64_t* flip = flipw + g * W;
    const int64_t v0 = voff[g], v1 = voff[g + 1];
    int P = 1;
    while (P < K) P <<= 1;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_min = 0x7FFFFFFF;
        s_ns = 0;
    }
    for (int i = tid; i < P; i += BC_THREADS) {
        key[i] = i < K ? hashes[g * KP + i] : ~0ull;
        idx[i] = i < K ? i : 0x7FFFFFFF;
        if (i < K) {
            cnt[i] = 0;
            state[i] = i;
        }
    }
    __syncthreads();
    // bitonic sort by (key, idx)
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += BC_THREADS) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[i] > key[p] || (key[i] == key[p] && idx[i] > idx[p]);
                    if (gt == up) {
                        const uint64_t tk = key[i];
                        key[i] = key[p];
                        key[p] = tk;
                        const int32_t ti = idx[i];
                        idx[i] = idx[p];
                        idx[p] = ti;
                    }
                }
            }
            __syncthreads();
        }
    // run leaders: inclusive max-scan of head positions
    for (int i = tid; i < K; i += BC_THREADS) lead[i] = (i == 0 || key[i] != key[i - 1]) ? i : -1;
    __syncthreads();
    for (int d = 1; d < K; d <<= 1) {
        int32_t tmp[BC_MAXK / BC_THREADS];
        int q = 0;
        for (int i = tid; i < K; i += BC_THREADS, q++) tmp[q] = (i >= d) ? max(lead[i], lead[i - d]) : lead[i];
        __syncthreads();
        q = 0;
        for (int i = tid; i < K; i += BC_THREADS, q++) lead[i] = tmp[q];
        __syncthreads();
    }
    // compare every non-leader with its leader (one warp per tree)
    const int warp = tid >> 5, nwarps = BC_THREADS / 32;
    for (int i = warp; i < K; i += nwarps) {
        const int li = lead[i];
        if (li == i) continue;
        const bool same = bc_same(lab, W, flip, v0, v1, idx[i], idx[li]);
        if ((tid & 31) == 0) state[idx[i]] = same ? idx[li] : -1;  // -1: differs (hash collision)
    }
    __syncthreads();
    // rare path: trees that differ from their leader, matched in sorted order
    // against the earlier differing trees of the same run
    if (warp == 0) {
        for (int i = 0; i < K; i++) {
            if (state[idx[i]] != -1) continue;
            int rep = idx[i];
            for (int j = lead[i] + 1; j < i; j++) {
                const int tj = idx[j];
                if (state[tj] == tj && bc_same(lab, W, flip, v0, v1, idx[i], tj)) {
                    rep = tj;
                    break;
                }
            }
            __syncwarp();
            if ((tid & 31) == 0) state[idx[i]] = rep;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = tid; t < K; t += BC_THREADS) {
        atomicAdd(&cnt[state[t]], 1);
        atomicMin(&s_min, counts[g * KP + t]);
    }
    __syncthreads();
    // output positions: representatives in tree order
    if (tid == 0) {
        int r = 0;
        for (int t = 0; t < K; t++) {
            rank[t] = (state[t] == t) ? r : -1;
            if (state[t] == t) r++;
        }
        s_ns = r;
    }
    __syncthreads();
    if (entries)
        for (int t = tid; t < K; t += BC_THREADS)
            if (state[t] == t) {
                sb_cloud_entry e;
                e.hash = hashes[g * KP + t];
                e.S = counts[g * KP + t];
                e.count = cnt[t];
                e.first_tree = *tree0p + t;
                entries[g * (int64_t)K + rank[t]] = e;
            }
    if (tid == 0) {
        nstates_out[g] = s_ns;
        frmin_out[g] = s_min;
    }
}

extern "C" sb_status sb_batch_cloud(sb_ctx* c, int32_t* n_states_out, int32_t* fr_min_out, sb_cloud_entry* entries_out)
{
    if (!c || !n_states_out || !fr_min_out) return SB_ERR_ARG;
    if (!c->has_graph || c->batch_G <= 0) return sb_fail(c, SB_ERR_STATE, "no batch of graphs loaded");
    if (!c->has_batch) return sb_fail(c, SB_ERR_STATE, "no sampled trees");
    if (c->K > BC_MAXK) return sb_fail(c, SB_ERR_ARG, "batch clouds need K <= %d", BC_MAXK);
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_score_batch(c));
    const int64_t G = c->batch_G;
    int32_t* ns = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)G);
    int32_t* fm = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)G);
    sb_cloud_entry* ent = entries_out ? (sb_cloud_entry*)sb_dalloc(c, sizeof(sb_cloud_entry) * (size_t)G * c->K) : nullptr;
    sb_status st = SB_OK;
    if (!ns || !fm || (entries_out && !ent)) st = sb_fail(c, SB_ERR_OOM, "batch cloud output");
    if (st == SB_OK) {
        SbProf prof(c, SB_PROF_CLOUD);
        k_batch_cloud<<<(unsigned)G, BC_THREADS, 0, c->stream>>>(c->hashes, c->counts, 64 * (int64_t)c->W, (int)c->K,
                                                                sb_tree0_ptr(c->sync), c->labels, c->W, c->flipw,
                                                                c->b_voff, ns, fm, ent);
        st = sb_after_launch(c, "k_batch_cloud");
    }
    if (st == SB_OK) st = sb_copy_out(c, n_states_out, ns, sizeof(int32_t) * (size_t)G);
    if (st == SB_OK) st = sb_copy_out(c, fr_min_out, fm, sizeof(int32_t) * (size_t)G);
    if (st == SB_OK && ent) st = sb_copy_out(c, entries_out, ent, sizeof(sb_cloud_entry) * (size_t)G * c->K);
    cudaStreamSynchronize(c->stream);
    sb_dfree(c, ns);
    sb_dfree(c, fm);
    sb_dfree(c, ent);
    return st;
}

// per-graph clouds of the current batch's trees into device arrays (no
// entries, no host synchronisation): the cloud step of sb_batch_steps
sb_status sb_batch_cloud_enqueue(sb_ctx* c, int32_t* n_states, int32_t* fr_min)
{
    SbProf prof(c, SB_PROF_CLOUD);
    k_batch_cloud<<<(unsigned)c->batch_G, BC_THREADS, 0, c->stream>>>(c->hashes, c->counts, 64 * (int64_t)c->W,
                                                                     (int)c->K, sb_tree0_ptr(c->sync), c->labels,
                                                                     c->W, c->flipw, c->b_voff, n_states, fr_min,
                                                                     nullptr);
    return sb_after_launch(c, "k_batch_cloud");
}
