// sb_ctx.cu -- context lifetime, errors, memory, and the two device
// primitives the ingest path needs: an exclusive scan and an LSD radix sort.
#include <stdarg.h>
#include <stdlib.h>

#include <new>

#include "sb_internal.cuh"

// ------------------------------------------------------------------ errors
sb_status sb_fail(sb_ctx* c, sb_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

sb_status sb_cuda_fail(sb_ctx* c, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return sb_fail(c, SB_ERR_OOM, "out of device memory at %s", where);
    }
    return sb_fail(c, SB_ERR_CUDA, "CUDA error %s (%s) at %s", cudaGetErrorName(e), cudaGetErrorString(e), where);
}

sb_status sb_after_launch(sb_ctx* c, const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sb_cuda_fail(c, e, what);
    c->prof_launch[c->cur_family]++;
    return SB_OK;
}

// ---------------------------------------------------------------- profiling
static cudaEvent_t ev_get(sb_ctx* c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void sb_prof_begin(sb_ctx* c, cudaEvent_t* a)
{
    *a = nullptr;
    if (!c->prof_on || c->capturing || c->prof_recs.size() > 200000) return;
    *a = ev_get(c);
    if (*a) cudaEventRecord(*a, c->stream);
}

void sb_prof_end(sb_ctx* c, int fam, cudaEvent_t a)
{
    if (!a) return;
    cudaEvent_t b = ev_get(c);
    if (!b) {
        c->ev_pool.push_back(a);
        return;
    }
    cudaEventRecord(b, c->stream);
    c->prof_recs.push_back({a, b, fam});
}

extern "C" sb_status sb_profile(sb_ctx* c, int enable)
{
    if (!c) return SB_ERR_ARG;
    c->prof_on = enable ? 1 : 0;
    return SB_OK;
}

extern "C" sb_status sb_profile_read(sb_ctx* c, double* ms_out, int64_t* launches_out)
{
    if (!c) return SB_ERR_ARG;
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    for (const sb_prof_rec& r : c->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->prof_ms[r.fam] += ms;
        else cudaGetLastError();
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    for (int i = 0; i < SB_PROF_N; i++) {
        if (ms_out) ms_out[i] = c->prof_ms[i];
        if (launches_out) launches_out[i] = c->prof_launch[i];
        c->prof_ms[i] = 0.0;
        c->prof_launch[i] = 0;
    }
    return SB_OK;
}

extern "C" const char* sb_status_str(sb_status s)
{
    switch (s) {
    case SB_OK: return "ok";
    case SB_ERR_ARG: return "invalid argument";
    case SB_ERR_CUDA: return "CUDA error";
    case SB_ERR_OOM: return "out of memory";
    case SB_ERR_SELF_LOOP: return "self-loop in input";
    case SB_ERR_BAD_SIGN: return "edge sign not +1/-1";
    case SB_ERR_INCONSISTENT: return "vertex pair with both signs";
    case SB_ERR_DUPLICATE: return "duplicate vertex pair";
    case SB_ERR_DISCONNECTED: return "graph is not connected";
    case SB_ERR_RANGE: return "vertex id out of range";
    case SB_ERR_STATE: return "call out of order";
    case SB_ERR_CLOUD_FULL: return "frustration cloud full";
    case SB_ERR_TIMEOUT: return "device wait timed out";
    case SB_ERR_DEVICE_CHECK: return "device consistency check failed";
    default: return "unknown status";
    }
}

extern "C" const char* sb_last_error(const sb_ctx* c) { return c ? c->err : "no context"; }

// ------------------------------------------------------------------ memory
void* sb_dalloc(sb_ctx* c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->alloc) return c->alloc(bytes, (void*)c->stream, c->alloc_user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void sb_dfree(sb_ctx* c, void* p)
{
    if (!p) return;
    if (c->free_fn) c->free_fn(p, (void*)c->stream, c->alloc_user);
    else cudaFree(p);
}

sb_status sb_ensure(sb_ctx* c, void** p, size_t* cap, size_t bytes)
{
    if (*p && *cap >= bytes) return SB_OK;
    sb_dfree(c, *p);
    *p = nullptr;
    *cap = 0;
    void* q = sb_dalloc(c, bytes);
    if (!q) return sb_fail(c, SB_ERR_OOM, "device allocation of %zu bytes failed", bytes);
    *p = q;
    *cap = bytes;
    return SB_OK;
}

bool sb_is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sb_status sb_copy_out(sb_ctx* c, void* dst, const void* src_dev, size_t bytes)
{
    if (bytes == 0 || !dst) return SB_OK;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, c->stream));
    if (!sb_is_device_ptr(dst)) SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    return SB_OK;
}

#define SB_FREE(field)           \
    do {                         \
        sb_dfree(c, (c)->field); \
        (c)->field = nullptr;    \
    } while (0)

void sb_release_batch(sb_ctx* c)
{
    SB_FREE(labels);
    c->labels_cap = 0;
    SB_FREE(flipw);
    c->flipw_cap = 0;
    SB_FREE(hashes);
    c->hashes_cap = 0;
    SB_FREE(hwsum);
    c->hwsum_cap = 0;
    SB_FREE(counts);
    c->counts_cap = 0;
    SB_FREE(vis);
    SB_FREE(fr0);
    SB_FREE(fr1);
    SB_FREE(done);
    SB_FREE(hubnew);
    SB_FREE(hubbest);
    SB_FREE(mst_P);
    SB_FREE(mst_R);
    SB_FREE(mst_Y);
    SB_FREE(mst_L);
    SB_FREE(mst_B);
    SB_FREE(mst_win);
    SB_FREE(mst_flags);
    c->mst_cap = 0;
    c->labels_cap = 0;
    c->bfs_cap_words = 0;
    c->has_batch = false;
}

void sb_release_cloud(sb_ctx* c)
{
    SB_FREE(cl_table);
    SB_FREE(cl_entries);
    SB_FREE(cl_bits);
    SB_FREE(cl_meta);
    SB_FREE(cl_assign);
    SB_FREE(cl_rep);
    SB_FREE(cl_mismatch);
    SB_FREE(cl_touch);
    c->cl_slots = 0;
    c->cl_n_host = 0;
    c->cl_order.clear();
}

void sb_release_graphl(sb_ctx* c)
{
    SB_FREE(gl_partial);
    SB_FREE(gl_red);
    SB_FREE(gl_buf);
    SB_FREE(gl_scale);
    SB_FREE(gl_colmax);
    SB_FREE(gl_misc);
    if (c->gl_exec) cudaGraphExecDestroy(c->gl_exec);
    c->gl_exec = nullptr;
    memset(c->gl_exec_key, 0, sizeof(c->gl_exec_key));
    c->gl_partial_cap = c->gl_red_cap = c->gl_buf_cap = c->gl_misc_cap = 0;
    c->gl_scale_cap = c->gl_colmax_cap = 0;
}

void sb_release_graph(sb_ctx* c)
{
    sb_release_batch(c);
    sb_release_cloud(c);
    SB_FREE(edges);
    SB_FREE(sc_edges);
    SB_FREE(rowptr);
    SB_FREE(col);
    SB_FREE(items);
    SB_FREE(hub_vertex);
    SB_FREE(gl_items);
    SB_FREE(gl_hub_first);
    SB_FREE(gl_hub_vertex);
    SB_FREE(gl_hub_count);
    SB_FREE(vweight);
    if (c->gl_exec) cudaGraphExecDestroy(c->gl_exec);
    c->gl_exec = nullptr;
    memset(c->gl_exec_key, 0, sizeof(c->gl_exec_key));
    SB_FREE(bs_frmin);
    SB_FREE(bs_fm);
    SB_FREE(bs_ns);
    c->bs_cap = 0;
    if (c->bs_exec) cudaGraphExecDestroy(c->bs_exec);
    c->bs_exec = nullptr;
    memset(c->bs_exec_key, 0, sizeof(c->bs_exec_key));
    c->graph_gen++;
    SB_FREE(b_voff);
    SB_FREE(b_eoff);
    SB_FREE(vgid);
    SB_FREE(vgoff);
    c->batch_G = 0;
    c->h_voff.clear();
    c->h_eoff.clear();
    c->has_graph = false;
    c->n = c->m = c->n_items = c->n_hubs = 0;
    c->n_gl_items = c->n_gl_hubs = c->n_gl_partials = 0;
}

// ----------------------------------------------------------------- context
extern "C" sb_status sb_create(sb_ctx** out, int device, void* cuda_stream)
{
    if (!out) return SB_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SB_ERR_ARG;
    }
    sb_ctx* c = new (std::nothrow) sb_ctx();
    if (!c) return SB_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SB_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, device) != cudaSuccess || c->clock_khz <= 0) {
        cudaGetLastError();
        c->clock_khz = 2070000;  // the GB300's largest SM clock
    }
    *out = c;
    return SB_OK;
}

extern "C" void sb_destroy(sb_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    sb_release_graph(c);
    sb_release_graphl(c);
    sb_dfree(c, c->sync);
    sb_dfree(c, c->tmp);
    for (const sb_prof_rec& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_in) cudaEventDestroy(c->cap_in);
    if (c->cap_out) cudaEventDestroy(c->cap_out);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

extern "C" sb_status sb_set_allocator(sb_ctx* c, sb_alloc_fn alloc, sb_free_fn free_fn, void* user)
{
    if (!c || (!alloc) != (!free_fn)) return SB_ERR_ARG;
    if (c->has_graph || c->gl_buf || c->sync)
        return sb_fail(c, SB_ERR_STATE, "sb_set_allocator must precede any allocation");
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->alloc_user = user;
    return SB_OK;
}

extern "C" sb_status sb_set_tuning(sb_ctx* c, int32_t knob, int64_t value)
{
    if (!c || knob < 0 || knob >= SB_TUNE_N || value < 0) return SB_ERR_ARG;
    if (knob == SB_TUNE_BFS_WORDS && value > SB_WORDS_MAX) return sb_fail(c, SB_ERR_ARG, "at most 32 words per launch");
    if (knob == SB_TUNE_SCORE_BLOCKS_SM && value > 32) return sb_fail(c, SB_ERR_ARG, "at most 32 blocks per SM");
    if (knob == SB_TUNE_GL_LANES && value != 0 && value != 8 && value != 16 && value != 32)
        return sb_fail(c, SB_ERR_ARG, "graphL lanes must be 8, 16 or 32");
    if (knob == SB_TUNE_BFS_GROUP && (value > 32 || (value & (value - 1)) != 0))
        return sb_fail(c, SB_ERR_ARG, "BFS group must be a power of two <= 32");
    if (knob == SB_TUNE_WAIT_US && value > 60000000) return sb_fail(c, SB_ERR_ARG, "wait limit at most 6e7 us");
    if (knob == SB_TUNE_STALL_TEST && value > 1) return sb_fail(c, SB_ERR_ARG, "stall test is 0 or 1");
    if (knob == SB_TUNE_MST_WORDS && value > SB_TREES_MAX / 64)
        return sb_fail(c, SB_ERR_ARG, "at most %d Kruskal words per pass", SB_TREES_MAX / 64);
    c->tune[knob] = value;
    return SB_OK;
}

long long sb_wait_cycles(const sb_ctx* c)
{
    const long long us = c->tune[SB_TUNE_WAIT_US] > 0 ? (long long)c->tune[SB_TUNE_WAIT_US] : SB_WAIT_DEFAULT_US;
    return us * (long long)c->clock_khz / 1000;
}

extern "C" sb_status sb_get_tuning(sb_ctx* c, int32_t knob, int64_t* value)
{
    if (!c || !value || knob < 0 || knob >= SB_TUNE_N) return SB_ERR_ARG;
    *value = c->tune[knob];
    return SB_OK;
}

extern "C" sb_status sb_sync(sb_ctx* c)
{
    if (!c) return SB_ERR_ARG;
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    SB_CHECK_CUDA(c, cudaGetLastError());
    if (c->sync) {
        // errors that sb_batch_steps left on the device
        uint32_t sticky = 0;
        SB_CHECK_CUDA(c, cudaMemcpy(&sticky, c->sync + 34, sizeof(sticky), cudaMemcpyDeviceToHost));
        if (sticky) {
            SB_CHECK_CUDA(c, cudaMemset(c->sync + 34, 0, sizeof(uint32_t)));
            if (sticky & 1u) return sb_fail(c, SB_ERR_TIMEOUT, "a bounded device wait gave up during the steps");
            return sb_fail(c, SB_ERR_DEVICE_CHECK, "a device-side check failed during the steps");
        }
    }
    return SB_OK;
}

// -------------------------------------------------------------------- scan
#define SCAN_THREADS 256
#define SCAN_ITEMS 8
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

// exclusive scan inside one tile; tile totals to sums[]
__global__ void k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                            int32_t* __restrict__ sums)
{
    __shared__ int32_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t k = base + i;
        v[i] = k < n ? in[k] : 0;
        run += v[i];
    }
    // inclusive scan of per-thread totals across the block
    int32_t x = run;
    unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int32_t wofs = 0;
    for (unsigned w = 0; w < warp; w++) wofs += warp_tot[w];
    int32_t excl = wofs + x - run;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t k = base + i;
        if (k < n) out[k] = excl;
        excl += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = wofs + x;
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ ofs)
{
    int64_t k = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int32_t o = ofs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++, k += SCAN_THREADS)
        if (k < n) out[k] += o;
}

__global__ void k_scan_total(const int32_t* in, const int32_t* out, int64_t n, int64_t* total)
{
    *total = n > 0 ? (int64_t)out[n - 1] + (int64_t)in[n - 1] : 0;
}

sb_status sb_scan_i32(sb_ctx* c, const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev)
{
    if (n <= 0) {
        if (total_dev) SB_CHECK_CUDA(c, cudaMemsetAsync(total_dev, 0, sizeof(int64_t), c->stream));
        return SB_OK;
    }
    int64_t tiles = sb_cdiv(n, SCAN_TILE);
    int32_t* sums = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)tiles);
    int32_t* sofs = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)tiles);
    if (!sums || !sofs) {
        sb_dfree(c, sums);
        sb_dfree(c, sofs);
        return sb_fail(c, SB_ERR_OOM, "scan scratch");
    }
    sb_status st = SB_OK;
    k_scan_tile<<<(unsigned)tiles, SCAN_THREADS, 0, c->stream>>>(in, out, n, sums);
    st = sb_after_launch(c, "k_scan_tile");
    if (st == SB_OK && tiles > 1) {
        st = sb_scan_i32(c, sums, sofs, tiles, nullptr);
        if (st == SB_OK) {
            k_scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, c->stream>>>(out, n, sofs);
            st = sb_after_launch(c, "k_scan_add");
        }
    }
    if (st == SB_OK && total_dev) {
        k_scan_total<<<1, 1, 0, c->stream>>>(in, out, n, total_dev);
        st = sb_after_launch(c, "k_scan_total");
    }
    sb_dfree(c, sums);
    sb_dfree(c, sofs);
    return st;
}

// -------------------------------------------------------------- radix sort
#define RS_THREADS 256
#define RS_ITEMS 16
#define RS_TILE (RS_THREADS * RS_ITEMS)
#define RS_WARPS (RS_THREADS / 32)

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
                             int64_t ntiles)
{
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t k = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: keys of a tile are taken in input order (striped rounds,
// lane order inside a warp, warp order inside a round).
__global__ void k_radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n, int shift,
                                const int32_t* __restrict__ ofs, int64_t ntiles)
{
    __shared__ int32_t running[256];
    __shared__ int32_t wcnt[RS_WARPS][256];
    unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5;
    running[t] = ofs[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) wcnt[w][t] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t k = base + (int64_t)i * RS_THREADS + t;
        bool valid = k < n;
        uint64_t key = valid ? in[k] : 0;
        unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int32_t pre = 0;
            for (unsigned w = 0; w < warp; w++) pre += wcnt[w][d];
            out[running[d] + pre + rank] = key;
        }
        __syncthreads();
        int32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            add += wcnt[w][t];
            wcnt[w][t] = 0;
        }
        running[t] += add;
        __syncthreads();
    }
}

sb_status sb_radix_sort_u64(sb_ctx* c, uint64_t* keys, int64_t n, int bits)
{
    if (n <= 1 || bits <= 0) return SB_OK;
    int64_t ntiles = sb_cdiv(n, RS_TILE);
    int64_t hn = 256 * ntiles;
    uint64_t* alt = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)n);
    int32_t* hist = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)hn);
    int32_t* ofs = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)hn);
    sb_status st = SB_OK;
    if (!alt || !hist || !ofs) st = sb_fail(c, SB_ERR_OOM, "radix sort scratch");
    uint64_t* src = keys;
    uint64_t* dst = alt;
    for (int shift = 0; st == SB_OK && shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, c->stream>>>(src, n, shift, hist, ntiles);
        st = sb_after_launch(c, "k_radix_hist");
        if (st == SB_OK) st = sb_scan_i32(c, hist, ofs, hn, nullptr);
        if (st == SB_OK) {
            k_radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, c->stream>>>(src, dst, n, shift, ofs, ntiles);
            st = sb_after_launch(c, "k_radix_scatter");
        }
        uint64_t* tswap = src;
        src = dst;
        dst = tswap;
    }
    if (st == SB_OK && src != keys)
        if (cudaMemcpyAsync(keys, src, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess)
            st = sb_cuda_fail(c, cudaGetLastError(), "radix copy back");
    sb_dfree(c, alt);
    sb_dfree(c, hist);
    sb_dfree(c, ofs);
    return st;
}
