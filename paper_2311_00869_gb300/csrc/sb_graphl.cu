// sb_graphl.cu -- graphL (Sec. 4, Alg. 2): relaxed loss (Eq. 3), discrete
// loss (Eq. 2), the adjoint dL/dG_v = -1/2 sum_j e_vj G_j (Eq. 4), the descent
// update G <- G - alpha dL/dG, and the final rounding (Algorithm 2).
//
// Layout: G is n x R float32, row-major (the R starting points of one vertex
// are contiguous), so a neighbour gather reads a contiguous row segment.
// Determinism: the adjoint sums each CSR row in a fixed order (blocks of 32
// neighbours, then across blocks; rows longer than SB_GL_CHUNK are cut into
// chunks whose partial sums are added in chunk order by a second kernel).
// Integer counts and column maxima use order-free atomics; float sums never do.
#include <algorithm>

#include "sb_internal.cuh"

#define GL_THREADS 256
#define GL_ROWS_MIN_BLOCKS 4  // blocks per SM the row kernel's registers must allow

struct GlArgs {
    const sb_bfs_item* items;   // chunks of split rows first, then whole rows
    int64_t n_items;
    int64_t n_split_items;      // items [0, n_split_items) are chunks of split rows
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* hub_first;
    const float* gin;      // n x R input
    float* gout_rows;      // n x R output
    float* partial;        // partial sums of split rows
    const float* upstream; // GRAD: gout[G x R] (G = 1 for one graph)
    const float* scale;    // STEP: input scale per (graph, column), a power of two
    float half_alpha;      // STEP: alpha / 2
    int32_t* F;            // STEP: discrete-loss accumulator (x2) per (graph, column), nullable
    uint32_t* colmax;      // STEP: max |G_out| bits per (graph, column)
    const int32_t* vgid;   // graph of each vertex in a batch, or null (one graph)
    int64_t n;
    int R;
};

template <int VEC> struct Vec;
template <> struct Vec<1> {
    typedef float T;
    static __device__ __forceinline__ T ld(const float* p) { return __ldg(p); }
};
template <> struct Vec<4> {
    typedef float4 T;
    static __device__ __forceinline__ T ld(const float* p) { return __ldg((const float4*)p); }
};

__device__ __forceinline__ float flip_sign(float x, uint32_t negbit) { return __uint_as_float(__float_as_uint(x) ^ negbit); }
// theta = -1 exactly when G < 0 (so -0.0 rounds to +1, as G >= 0 does)
__device__ __forceinline__ uint32_t is_neg(float x) { return __float_as_uint(x) > 0x80000000u ? 1u : 0u; }

// Per-lane running column max / frustrated-edge count of one graph; flushed
// into the block's shared accumulators (one graph) or into the per-(graph,
// column) global accumulators (a batch) when the graph changes.
template <int VEC>
struct GlCols {
    int64_t g = -1;
    uint32_t mx[VEC];
    int32_t fc[VEC];
    __device__ __forceinline__ void reset(int64_t gg)
    {
        g = gg;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            mx[k] = 0;
            fc[k] = 0;
        }
    }
    __device__ __forceinline__ void flush(const GlArgs& A, int r0, int32_t* sF, uint32_t* smax)
    {
        if (g < 0) return;
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const int r = r0 + k;
            if (r >= A.R) continue;
            if (!A.vgid) {
                if (mx[k]) atomicMax(smax + r, mx[k]);
                if (fc[k]) atomicAdd(sF + r, fc[k]);
            } else {
                if (mx[k]) atomicMax(A.colmax + g * A.R + r, mx[k]);
                if (fc[k] && A.F) atomicAdd(A.F + g * A.R + r, fc[k]);
            }
        }
    }
};

// epilogue shared by whole rows and by combined split rows; returns |G_out| bits
template <bool STEP>
__device__ __forceinline__ uint32_t gl_emit(const GlArgs& A, int64_t v, int64_t g, int r, float acc)
{
    const int64_t idx = v * A.R + r;
    if (!STEP) {
        A.gout_rows[idx] = -0.5f * A.upstream[g * A.R + r] * acc;  // gout is G x R in a batch
        return 0u;
    }
    const float sc = A.scale[g * A.R + r];
    const float x = A.gin[idx] * sc;
    const float out = x + A.half_alpha * (acc * sc);
    A.gout_rows[idx] = out;
    return __float_as_uint(fabsf(out));
}

// Rows (and chunks of split rows): a sub-warp of SL lanes per (item, segment
// of SL*VEC columns).  The segments run one after the other over the whole
// grid, so one segment's columns of G (n x SL*VEC floats; 84 MB for 656k
// vertices at 32 columns) stay in L2 while every row gathers from them.
// Within a segment the sub-warps take blocks of GL_ITEM_BLOCK consecutive
// items in turn: the chunks of one long row spread over many sub-warps, and a
// block (rows in vertex order) rarely crosses a graph of a batch.
#define GL_ITEM_BLOCK 16
template <int VEC, int SL, bool STEP>
__global__ void __launch_bounds__(GL_THREADS, GL_ROWS_MIN_BLOCKS) k_gl_rows(GlArgs A)
{
    extern __shared__ uint32_t gsm[];
    int32_t* sF = (int32_t*)gsm;  // R
    uint32_t* smax = gsm + A.R;   // R
    const int R = A.R;
    if (STEP) {
        for (int i = threadIdx.x; i < R; i += GL_THREADS) {
            sF[i] = 0;
            smax[i] = 0;
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int sl = lane & (SL - 1);
    const unsigned smask = SL == 32 ? 0xffffffffu : (((1u << SL) - 1u) << (lane & ~(SL - 1)));
    const int64_t subs_total = (int64_t)gridDim.x * (GL_THREADS / SL);
    const int64_t sub_id = (int64_t)blockIdx.x * (GL_THREADS / SL) + threadIdx.x / SL;
    constexpr int seg_w = SL * VEC;
    const int nseg = (R + seg_w - 1) / seg_w;
    // split-row chunks one at a time, then whole rows by blocks: work unit w
    // covers items [lo(w), hi(w))
    const int64_t nsplit = A.n_split_items;
    const int64_t nunits = nsplit + sb_cdiv(A.n_items - nsplit, GL_ITEM_BLOCK);
    const bool wantF = STEP && A.F != nullptr;
    for (int seg = 0; seg < nseg; seg++) {
        const int r0 = seg * seg_w + sl * VEC;
        const bool act = r0 < R;
        GlCols<VEC> cols;
        for (int64_t wu = sub_id; wu < nunits; wu += subs_total)
        for (int64_t it = wu < nsplit ? wu : nsplit + (wu - nsplit) * GL_ITEM_BLOCK,
                     it_end = wu < nsplit ? wu + 1 : min(A.n_items, nsplit + (wu - nsplit + 1) * GL_ITEM_BLOCK);
             it < it_end; it++) {
            const sb_bfs_item itm = A.items[it];
            const int64_t g = A.vgid ? A.vgid[itm.v] : 0;
            if (STEP && g != cols.g) {
                if (act) cols.flush(A, r0, sF, smax);
                cols.reset(g);
            }
            float acc[VEC], blk[VEC];
            int32_t fcnt[VEC];
            uint32_t sv[VEC];
#pragma unroll
            for (int k = 0; k < VEC; k++) {
                acc[k] = 0.f;
                fcnt[k] = 0;
                sv[k] = 0;
            }
            if (wantF && act) {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    sv[k] = (r0 + k < R) ? is_neg(A.gin[(int64_t)itm.v * R + r0 + k]) : 0u;
            }
            // blocks of 32 neighbours (fixed order), SL column ids loaded at a time
            for (int j0 = itm.beg; j0 < itm.end; j0 += 32) {
                const int cnt = min(32, itm.end - j0);
#pragma unroll
                for (int k = 0; k < VEC; k++) blk[k] = 0.f;
                for (int jj = 0; jj < cnt; jj += SL) {
                    const int cc_n = min(SL, cnt - jj);
                    const uint32_t mycol = sl < cc_n ? (uint32_t)__ldg(A.col + j0 + jj + sl) : 0u;
                    int q0 = 0;
                    if constexpr (VEC == 4) {
                        // four neighbour rows in flight, then added in order
                        for (; q0 + 4 <= cc_n; q0 += 4) {
                            uint32_t cc[4];
                            float4 x[4];
#pragma unroll
                            for (int i = 0; i < 4; i++) cc[i] = __shfl_sync(smask, mycol, q0 + i, SL);
                            if (act) {
#pragma unroll
                                for (int i = 0; i < 4; i++)
                                    x[i] = Vec<4>::ld(A.gin + (int64_t)(cc[i] & SB_ID_MASK) * R + r0);
#pragma unroll
                                for (int i = 0; i < 4; i++) {
                                    const uint32_t nb = cc[i] & 0x80000000u, nb1 = cc[i] >> 31;
                                    blk[0] += flip_sign(x[i].x, nb);
                                    blk[1 % VEC] += flip_sign(x[i].y, nb);
                                    blk[2 % VEC] += flip_sign(x[i].z, nb);
                                    blk[3 % VEC] += flip_sign(x[i].w, nb);
                                    if (wantF) {
                                        fcnt[0] += (int)(is_neg(x[i].x) ^ nb1 ^ sv[0]);
                                        fcnt[1 % VEC] += (int)(is_neg(x[i].y) ^ nb1 ^ sv[1 % VEC]);
                                        fcnt[2 % VEC] += (int)(is_neg(x[i].z) ^ nb1 ^ sv[2 % VEC]);
                                        fcnt[3 % VEC] += (int)(is_neg(x[i].w) ^ nb1 ^ sv[3 % VEC]);
                                    }
                                }
                            }
                        }
                    }
                    for (int q = q0; q < cc_n; q++) {
                        const uint32_t cc = __shfl_sync(smask, mycol, q, SL);
                        const uint32_t nb = cc & 0x80000000u;
                        const uint32_t nb1 = cc >> 31;
                        const int64_t base = (int64_t)(cc & SB_ID_MASK) * R + r0;
                        if (act) {
                            if constexpr (VEC == 4) {
                                const float4 x = Vec<4>::ld(A.gin + base);
                                blk[0] += flip_sign(x.x, nb);
                                blk[1 % VEC] += flip_sign(x.y, nb);
                                blk[2 % VEC] += flip_sign(x.z, nb);
                                blk[3 % VEC] += flip_sign(x.w, nb);
                                if (wantF) {
                                    fcnt[0] += (int)(is_neg(x.x) ^ nb1 ^ sv[0]);
                                    fcnt[1 % VEC] += (int)(is_neg(x.y) ^ nb1 ^ sv[1 % VEC]);
                                    fcnt[2 % VEC] += (int)(is_neg(x.z) ^ nb1 ^ sv[2 % VEC]);
                                    fcnt[3 % VEC] += (int)(is_neg(x.w) ^ nb1 ^ sv[3 % VEC]);
                                }
                            } else {
                                const float x = Vec<1>::ld(A.gin + base);
                                blk[0] += flip_sign(x, nb);
                                if (wantF) fcnt[0] += (int)(is_neg(x) ^ nb1 ^ sv[0]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < VEC; k++) acc[k] += blk[k];
            }
            if (!act) continue;
            if (wantF) {
#pragma unroll
                for (int k = 0; k < VEC; k++) cols.fc[k] += fcnt[k];
            }
            if (itm.hub >= 0) {
                const int64_t slot = A.hub_first[itm.hub] + (itm.beg - A.rowptr[itm.v]) / SB_GL_CHUNK;
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (r0 + k < R) A.partial[slot * R + r0 + k] = acc[k];
            } else {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (r0 + k < R) {
                        const uint32_t b = gl_emit<STEP>(A, itm.v, g, r0 + k, acc[k]);
                        if (STEP) cols.mx[k] = max(cols.mx[k], b);
                    }
            }
        }
        if (STEP && act) cols.flush(A, r0, sF, smax);
    }
    if (STEP) {
        __syncthreads();
        if (!A.vgid)
            for (int i = threadIdx.x; i < R; i += GL_THREADS) {
                if (A.F && sF[i]) atomicAdd(A.F + i, sF[i]);
                if (smax[i]) atomicMax(A.colmax + i, smax[i]);
            }
    }
}

// Split rows: add chunk partials in chunk order, then the same epilogue.
template <bool STEP>
__global__ void __launch_bounds__(GL_THREADS) k_gl_combine(GlArgs A, const int32_t* __restrict__ hub_vertex,
                                                           const int32_t* __restrict__ hub_count, int64_t n_hubs)
{
    extern __shared__ uint32_t gsm[];
    uint32_t* smax = gsm + A.R;
    const int R = A.R;
    if (STEP) {
        for (int i = threadIdx.x; i < R; i += GL_THREADS) smax[i] = 0;
        __syncthreads();
    }
    const int64_t total = n_hubs * R;
    for (int64_t x = (int64_t)blockIdx.x * GL_THREADS + threadIdx.x; x < total; x += (int64_t)gridDim.x * GL_THREADS) {
        const int64_t h = x / R;
        const int r = (int)(x - h * R);
        const int64_t first = A.hub_first[h];
        const int cnt = hub_count[h];
        float acc = 0.f;
        for (int k = 0; k < cnt; k++) acc += A.partial[(first + k) * R + r];
        const int64_t v = hub_vertex[h];
        const int64_t g = A.vgid ? A.vgid[v] : 0;
        const uint32_t b = gl_emit<STEP>(A, v, g, r, acc);
        if (STEP && b) {
            if (A.vgid) atomicMax(A.colmax + g * R + r, b);
            else atomicMax(smax + r, b);
        }
    }
    if (STEP && !A.vgid) {
        __syncthreads();
        for (int i = threadIdx.x; i < R; i += GL_THREADS)
            if (smax[i]) atomicMax(A.colmax + i, smax[i]);
    }
}

// per-(graph, column) renorm decision and discrete-loss trace after one step
__global__ void k_gl_step_final(int64_t GR, uint32_t* colmax, int32_t* Facc, int32_t* F_trace_row, float* scale,
                                int32_t* exps, int renorm_log2)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < GR; r += (int64_t)gridDim.x * blockDim.x) {
        if (F_trace_row) F_trace_row[r] = Facc[r] / 2;
        Facc[r] = 0;
        const float mx = __uint_as_float(colmax[r]);
        colmax[r] = 0;
        float sc = 1.0f;
        if (renorm_log2 > 0 && mx >= ldexpf(1.0f, renorm_log2)) {
            sc = ldexpf(1.0f, -renorm_log2);
            exps[r] += renorm_log2;
        }
        scale[r] = sc;
    }
}

__global__ void k_gl_fill(float* p, int64_t n, float v)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) p[r] = v;
}

__global__ void k_gl_apply_scale(float* g, int64_t n, int R, const float* scale, const int32_t* vgid)
{
    const int64_t total = n * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / R;
        const int r = (int)(i - v * R);
        g[i] *= scale[(vgid ? (int64_t)vgid[v] : 0) * R + r];
    }
}

// Edge-parallel forward: per column r, Kahan sums of e_uv G_u G_v over the
// block's contiguous edge range, and the count of frustrated edges under
// theta = sign(G) (>= 0 -> +1).  Partials per block, summed in block order.
__global__ void __launch_bounds__(GL_THREADS) k_gl_fwd(const int2* __restrict__ edges, int64_t m,
                                                       const float* __restrict__ g, int R, double* __restrict__ red,
                                                       int32_t* __restrict__ Facc)
{
    const int64_t per = sb_cdiv(m, (int64_t)gridDim.x);
    const int64_t e0 = (int64_t)blockIdx.x * per, e1 = min(m, e0 + per);
    for (int r = threadIdx.x; r < R; r += GL_THREADS) {
        float s = 0.f, comp = 0.f;
        int32_t f = 0;
        for (int64_t e = e0; e < e1; e++) {
            const int2 ed = edges[e];
            const uint32_t nb = (uint32_t)ed.y & 0x80000000u;
            const float a = g[(int64_t)ed.x * R + r];
            const float b = g[(int64_t)((uint32_t)ed.y & SB_ID_MASK) * R + r];
            const float p = flip_sign(a * b, nb);
            // Kahan-Babuska (Neumaier) compensated sum
            const float t = s + p;
            comp += fabsf(s) >= fabsf(p) ? (s - t) + p : (p - t) + s;
            s = t;
            f += (int32_t)(is_neg(a) ^ is_neg(b) ^ (nb >> 31));
        }
        red[(int64_t)blockIdx.x * R + r] = (double)s + (double)comp;
        if (f) atomicAdd(Facc + r, f);
    }
}

__global__ void k_gl_fwd_final(const double* __restrict__ red, int nblocks, int R, int64_t m, float* loss,
                               int32_t* Facc, int32_t* F_out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; b++) s += red[(int64_t)b * R + r];
        loss[r] = (float)(0.5 * (double)m - 0.5 * s);
        if (F_out) F_out[r] = Facc[r];
        Facc[r] = 0;
    }
}

// Alg. 2 rounding: 64 edges per word; flips bit-packed per start point.
__global__ void __launch_bounds__(GL_THREADS) k_gl_round(const int2* __restrict__ edges, int64_t m,
                                                         const float* __restrict__ g, int R, int32_t* Facc,
                                                         uint64_t* flips, const int32_t* __restrict__ vgid)
{
    const int64_t nw = sb_cdiv(m, 64);
    for (int64_t w = blockIdx.x; w < nw; w += gridDim.x) {
        const int64_t e0 = w * 64;
        const int cnt = (int)min((int64_t)64, m - e0);
        for (int r = threadIdx.x; r < R; r += GL_THREADS) {
            uint64_t bits = 0;
            int64_t gcur = -1;
            int32_t fr = 0;
            for (int k = 0; k < cnt; k++) {
                const int2 ed = edges[e0 + k];
                const int64_t ge = vgid ? vgid[ed.x] : 0;
                if (ge != gcur) {  // frustrated edges are counted per graph
                    if (fr) atomicAdd(Facc + gcur * R + r, fr);
                    fr = 0;
                    gcur = ge;
                }
                const uint32_t a = is_neg(g[(int64_t)ed.x * R + r]);
                const uint32_t b = is_neg(g[(int64_t)((uint32_t)ed.y & SB_ID_MASK) * R + r]);
                const uint32_t f = a ^ b ^ ((uint32_t)ed.y >> 31);
                bits |= (uint64_t)f << k;
                fr += (int32_t)f;
            }
            if (flips) flips[(int64_t)r * nw + w] = bits;
            if (fr) atomicAdd(Facc + gcur * R + r, fr);
        }
    }
}

// Relaxed and discrete loss of every graph of a batch: one block per graph
// sums its own edges in order (Kahan-Babuska), so no cross-block reduction.
__global__ void __launch_bounds__(GL_THREADS) k_gl_fwd_graph(const int2* __restrict__ edges,
                                                             const int32_t* __restrict__ eoff,
                                                             const float* __restrict__ g, int R,
                                                             float* __restrict__ loss, int32_t* __restrict__ F)
{
    const int64_t gg = blockIdx.x;
    const int64_t e0 = eoff[gg], e1 = eoff[gg + 1];
    for (int r = threadIdx.x; r < R; r += GL_THREADS) {
        float s = 0.f, comp = 0.f;
        int32_t f = 0;
        for (int64_t e = e0; e < e1; e++) {
            const int2 ed = edges[e];
            const uint32_t nb = (uint32_t)ed.y & 0x80000000u;
            const float a = g[(int64_t)ed.x * R + r];
            const float b = g[(int64_t)((uint32_t)ed.y & SB_ID_MASK) * R + r];
            const float p = flip_sign(a * b, nb);
            const float t = s + p;
            comp += fabsf(s) >= fabsf(p) ? (s - t) + p : (p - t) + s;
            s = t;
            f += (int32_t)(is_neg(a) ^ is_neg(b) ^ (nb >> 31));
        }
        loss[gg * R + r] = (float)(0.5 * (double)(e1 - e0) - 0.5 * ((double)s + (double)comp));
        if (F) F[gg * R + r] = f;
    }
}

__global__ void k_gl_copy_F(int32_t* Facc, int64_t R, int32_t* out)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        if (out) out[r] = Facc[r];
        Facc[r] = 0;
    }
}

// ----------------------------------------------------------------- host
static sb_status gl_scratch(sb_ctx* c, int R, bool need_buf)
{
    SB_TRY(sb_ensure(c, (void**)&c->gl_partial, &c->gl_partial_cap,
                     sizeof(float) * (size_t)std::max<int64_t>(c->n_gl_partials, 1) * R));
    SB_TRY(sb_ensure(c, (void**)&c->gl_red, &c->gl_red_cap, sizeof(double) * (size_t)c->num_sms * 8 * R));
    const int64_t G = c->batch_G > 0 ? c->batch_G : 1;
    SB_TRY(sb_ensure(c, (void**)&c->gl_misc, &c->gl_misc_cap, sizeof(int32_t) * (size_t)G * R + 64));
    if (need_buf) SB_TRY(sb_ensure(c, (void**)&c->gl_buf, &c->gl_buf_cap, sizeof(float) * (size_t)c->n * R));
    return SB_OK;
}

static GlArgs gl_args(sb_ctx* c, int R)
{
    GlArgs A;
    memset(&A, 0, sizeof(A));
    A.items = c->gl_items;
    A.n_items = c->n_gl_items;
    A.n_split_items = c->n_gl_partials;
    A.rowptr = c->rowptr;
    A.col = c->col;
    A.hub_first = c->gl_hub_first;
    A.partial = c->gl_partial;
    A.n = c->n;
    A.R = R;
    A.vgid = c->batch_G > 0 ? c->vgid : nullptr;
    return A;
}

template <bool STEP>
static sb_status gl_rows_launch(sb_ctx* c, GlArgs& A)
{
    const bool vec4 = (A.R % 4 == 0) && (((uintptr_t)A.gin & 15) == 0);
    const int64_t lanes = c->tune[SB_TUNE_GL_LANES];
    const void* fn = !vec4        ? (const void*)k_gl_rows<1, 32, STEP>
                     : lanes == 32 ? (const void*)k_gl_rows<4, 32, STEP>
                     : lanes == 16 ? (const void*)k_gl_rows<4, 16, STEP>
                                   : (const void*)k_gl_rows<4, 8, STEP>;
    size_t smem = STEP ? sizeof(uint32_t) * 2 * (size_t)A.R : 0;
    if (smem > 48 * 1024) SB_CHECK_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SB_CHECK_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, GL_THREADS, smem));
    unsigned blocks = (unsigned)(c->num_sms * std::max(per_sm, 1));
    void* args[] = {&A};
    SbProf prof(c, SB_PROF_GL_ROWS);
    SB_CHECK_CUDA(c, cudaLaunchKernel(fn, dim3(blocks), dim3(GL_THREADS), args, smem, c->stream));
    SB_TRY(sb_after_launch(c, "k_gl_rows"));
    if (c->n_gl_hubs > 0) {
        const void* fc = (const void*)k_gl_combine<STEP>;
        if (smem > 48 * 1024)
            SB_CHECK_CUDA(c, cudaFuncSetAttribute(fc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int32_t* hv = c->gl_hub_vertex;
        const int32_t* hc = c->gl_hub_count;
        int64_t nh = c->n_gl_hubs;
        unsigned gb = (unsigned)std::min<int64_t>(sb_cdiv(nh * A.R, GL_THREADS), (int64_t)c->num_sms * 8);
        void* cargs[] = {&A, (void*)&hv, (void*)&hc, &nh};
        SB_CHECK_CUDA(c, cudaLaunchKernel(fc, dim3(gb), dim3(GL_THREADS), cargs, smem, c->stream));
        SB_TRY(sb_after_launch(c, "k_gl_combine"));
    }
    return SB_OK;
}

static sb_status gl_check(sb_ctx* c, int32_t R)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    if (R < 1 || R > 65536) return sb_fail(c, SB_ERR_ARG, "R must be in [1, 65536]");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    return SB_OK;
}

extern "C" sb_status sb_graphL_fwd(sb_ctx* c, const float* gamma, int32_t R, float* loss_out, int32_t* F_out)
{
    SB_TRY(gl_check(c, R));
    if (!gamma || !loss_out) return sb_fail(c, SB_ERR_ARG, "null pointer");
    SB_TRY(gl_scratch(c, R, false));
    if (c->batch_G > 0) {  // one block per graph; loss_out / F_out are G x R
        SbProf prof(c, SB_PROF_GL_FWD);
        k_gl_fwd_graph<<<(unsigned)c->batch_G, GL_THREADS, 0, c->stream>>>(c->edges, c->b_eoff, gamma, R, loss_out,
                                                                          F_out);
        return sb_after_launch(c, "k_gl_fwd_graph");
    }
    int32_t* Facc = c->gl_misc;
    SB_CHECK_CUDA(c, cudaMemsetAsync(Facc, 0, sizeof(int32_t) * R, c->stream));
    int nblocks = c->num_sms * 8;
    SbProf prof(c, SB_PROF_GL_FWD);
    k_gl_fwd<<<nblocks, GL_THREADS, 0, c->stream>>>(c->edges, c->m, gamma, R, c->gl_red, Facc);
    SB_TRY(sb_after_launch(c, "k_gl_fwd"));
    k_gl_fwd_final<<<(unsigned)sb_cdiv(R, 256), 256, 0, c->stream>>>(c->gl_red, nblocks, R, c->m, loss_out, Facc, F_out);
    return sb_after_launch(c, "k_gl_fwd_final");
}

extern "C" sb_status sb_graphL_bwd(sb_ctx* c, const float* gamma, int32_t R, const float* gout, float* grad_out)
{
    SB_TRY(gl_check(c, R));
    if (!gamma || !gout || !grad_out) return sb_fail(c, SB_ERR_ARG, "null pointer");
    SB_TRY(gl_scratch(c, R, false));
    GlArgs A = gl_args(c, R);
    A.gin = gamma;
    A.gout_rows = grad_out;
    A.upstream = gout;
    return gl_rows_launch<false>(c, A);
}

extern "C" sb_status sb_graphL_round(sb_ctx* c, const float* gamma, int32_t R, int32_t* F_out, uint64_t* flip_out)
{
    SB_TRY(gl_check(c, R));
    if (!gamma || !F_out) return sb_fail(c, SB_ERR_ARG, "null pointer");
    SB_TRY(gl_scratch(c, R, false));
    const int64_t GR = (c->batch_G > 0 ? c->batch_G : 1) * (int64_t)R;
    int32_t* Facc = c->gl_misc;
    SB_CHECK_CUDA(c, cudaMemsetAsync(Facc, 0, sizeof(int32_t) * GR, c->stream));
    unsigned blocks = (unsigned)std::min<int64_t>(std::max<int64_t>(sb_cdiv(c->m, 64), 1), (int64_t)c->num_sms * 8);
    SbProf prof(c, SB_PROF_GL_FWD);
    k_gl_round<<<blocks, GL_THREADS, 0, c->stream>>>(c->edges, c->m, gamma, R, Facc, flip_out,
                                                     c->batch_G > 0 ? c->vgid : nullptr);
    SB_TRY(sb_after_launch(c, "k_gl_round"));
    k_gl_copy_F<<<(unsigned)sb_cdiv(GR, 256), 256, 0, c->stream>>>(Facc, GR, F_out);
    return sb_after_launch(c, "k_gl_copy_F");
}

// Captures the descent loop into a CUDA graph (or reuses the captured one
// when the key matches) and launches it on c->stream.
static sb_status gl_descent_graph(sb_ctx* c, GlArgs& A, const uint64_t* key, const float* src, float* gamma_out,
                                  int steps, unsigned rb, int64_t GR, int32_t* Facc, int32_t* F_trace,
                                  int32_t* exps_out, int renorm_log2)
{
        const bool reuse = c->gl_exec && memcmp(key, c->gl_exec_key, sizeof(c->gl_exec_key)) == 0;
        if (!reuse) {
            if (c->gl_exec) cudaGraphExecDestroy(c->gl_exec);
            c->gl_exec = nullptr;
            cudaGraph_t graph = nullptr;
            SB_CHECK_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            c->capturing = true;
            sb_status st = SB_OK;
            const float* cur = src;
            for (int s = 0; s < steps && st == SB_OK; s++) {
                float* dst = (cur == gamma_out) ? c->gl_buf : gamma_out;
                A.gin = cur;
                A.gout_rows = dst;
                A.F = F_trace ? Facc : nullptr;
                st = gl_rows_launch<true>(c, A);
                if (st == SB_OK) {
                    k_gl_step_final<<<rb, 256, 0, c->stream>>>(GR, c->gl_colmax, Facc,
                                                               F_trace ? F_trace + (int64_t)s * GR : nullptr,
                                                               c->gl_scale, exps_out, renorm_log2);
                    st = sb_after_launch(c, "k_gl_step_final");
                }
                cur = dst;
            }
            c->capturing = false;
            cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
            if (st != SB_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ec != cudaSuccess) return sb_cuda_fail(c, ec, "cudaStreamEndCapture");
            ec = cudaGraphInstantiate(&c->gl_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) {
                c->gl_exec = nullptr;
                return sb_cuda_fail(c, ec, "cudaGraphInstantiate");
            }
            memcpy(c->gl_exec_key, key, sizeof(c->gl_exec_key));
        } else {
            // the kernels of a replay are counted like launched ones
            c->prof_launch[SB_PROF_GL_ROWS] += (int64_t)steps * (c->n_gl_hubs > 0 ? 2 : 1);
            c->prof_launch[SB_PROF_OTHER] += steps;
        }
        SbProf prof(c, SB_PROF_GL_ROWS);
        SB_CHECK_CUDA(c, cudaGraphLaunch(c->gl_exec, c->stream));
    return SB_OK;
}

extern "C" sb_status sb_graphL_descent(sb_ctx* c, const float* gamma0, float* gamma_out, int32_t R, float alpha,
                                       int32_t steps, int32_t renorm_log2, int32_t* exps_out, int32_t* F_trace,
                                       int32_t* F_final)
{
    SB_TRY(gl_check(c, R));
    if (!gamma0 || !gamma_out || !exps_out || steps < 0 || renorm_log2 < 0 || renorm_log2 > 100)
        return sb_fail(c, SB_ERR_ARG, "bad descent argument");
    SB_TRY(gl_scratch(c, R, true));
    const int64_t GR = (c->batch_G > 0 ? c->batch_G : 1) * (int64_t)R;  // per (graph, column)
    SB_TRY(sb_ensure(c, (void**)&c->gl_scale, &c->gl_scale_cap, sizeof(float) * (size_t)GR));
    SB_TRY(sb_ensure(c, (void**)&c->gl_colmax, &c->gl_colmax_cap, sizeof(uint32_t) * (size_t)GR));
    const size_t bytes = sizeof(float) * (size_t)c->n * R;
    int32_t* Facc = c->gl_misc;
    SB_CHECK_CUDA(c, cudaMemsetAsync(Facc, 0, sizeof(int32_t) * GR, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->gl_colmax, 0, sizeof(uint32_t) * GR, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(exps_out, 0, sizeof(int32_t) * GR, c->stream));
    unsigned rb = (unsigned)sb_cdiv(GR, 256);
    k_gl_fill<<<rb, 256, 0, c->stream>>>(c->gl_scale, GR, 1.0f);
    SB_TRY(sb_after_launch(c, "k_gl_fill"));
    const float* src = gamma0;
    if (gamma0 == gamma_out) {
        SB_CHECK_CUDA(c, cudaMemcpyAsync(c->gl_buf, gamma0, bytes, cudaMemcpyDeviceToDevice, c->stream));
        src = c->gl_buf;
    }
    GlArgs A = gl_args(c, R);
    A.scale = c->gl_scale;
    A.half_alpha = 0.5f * alpha;
    A.colmax = c->gl_colmax;
    // The step loop has no host synchronisation: it is captured once into a
    // CUDA graph and replayed while the call's buffers and parameters repeat.
    uint32_t abits;
    memcpy(&abits, &alpha, sizeof(abits));
    const uint64_t key[16] = {(uint64_t)(uintptr_t)src, (uint64_t)(uintptr_t)gamma_out, (uint64_t)R, abits,
                              (uint64_t)steps, (uint64_t)renorm_log2, (uint64_t)(uintptr_t)exps_out,
                              (uint64_t)(uintptr_t)F_trace, (uint64_t)(uintptr_t)c->gl_buf,
                              (uint64_t)(uintptr_t)c->gl_scale, (uint64_t)(uintptr_t)c->gl_partial,
                              (uint64_t)(uintptr_t)c->gl_misc, (uint64_t)(uintptr_t)c->gl_colmax,
                              (uint64_t)(uintptr_t)c->gl_items, (uint64_t)c->n,
                              1 + (uint64_t)c->tune[SB_TUNE_GL_LANES]};  // the captured kernels depend on it
    const float* last = src;
    for (int s = 0; s < steps; s++) last = (last == gamma_out) ? c->gl_buf : gamma_out;
    if (steps > 0) {
        // capture and replay on a private stream ordered after / before the
        // context stream (the legacy default stream cannot be captured)
        if (!c->cap_stream) {
            SB_CHECK_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            SB_CHECK_CUDA(c, cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming));
            SB_CHECK_CUDA(c, cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming));
        }
        cudaStream_t main_stream = c->stream;
        SB_CHECK_CUDA(c, cudaEventRecord(c->cap_in, main_stream));
        SB_CHECK_CUDA(c, cudaStreamWaitEvent(c->cap_stream, c->cap_in, 0));
        c->stream = c->cap_stream;
        sb_status stg = gl_descent_graph(c, A, key, src, gamma_out, steps, rb, GR, Facc, F_trace, exps_out,
                                         renorm_log2);
        c->stream = main_stream;
        SB_CHECK_CUDA(c, cudaEventRecord(c->cap_out, c->cap_stream));
        SB_CHECK_CUDA(c, cudaStreamWaitEvent(main_stream, c->cap_out, 0));
        SB_TRY(stg);
    }
    src = last;
    if (src != gamma_out) SB_CHECK_CUDA(c, cudaMemcpyAsync(gamma_out, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    // pending power-of-two scale of the last step
    unsigned gb = (unsigned)std::min<int64_t>(sb_cdiv((int64_t)c->n * R, 256), (int64_t)c->num_sms * 16);
    k_gl_apply_scale<<<gb, 256, 0, c->stream>>>(gamma_out, c->n, R, c->gl_scale, c->batch_G > 0 ? c->vgid : nullptr);
    SB_TRY(sb_after_launch(c, "k_gl_apply_scale"));
    if (F_final) SB_TRY(sb_graphL_round(c, gamma_out, R, F_final, nullptr));
    return SB_OK;
}

// ------------------------------------------- allocation-free relaxed loss
// sb_graphL_fwd_static runs the same two kernels as sb_graphL_fwd, but its
// scratch (per-block partial sums and the discrete-loss accumulators) lives in
// the fixed array below instead of context memory, so the call allocates
// nothing.  Every GPU that loads this library holds the array until the
// process exits.  All calls on a device share it and it keeps the last call's
// contents: the accumulators are cleared at the start of each call, and calls
// that overlap on the GPU (other streams, other host threads) race on it.
#define GL_STATIC_BLOCKS 304
#define GL_STATIC_RMAX 1024
static __device__ __align__(256) unsigned char g_gl_static_scratch[sizeof(double) * GL_STATIC_BLOCKS * GL_STATIC_RMAX +
                                                                   sizeof(int32_t) * GL_STATIC_RMAX];

#include <mutex>
static std::mutex g_static_mu;
static void* g_static_ptr[256];  // device address of the array, per device

extern "C" sb_status sb_graphL_fwd_static(const int32_t* edges, int64_t m, const float* gamma, int32_t R,
                                          float* loss_out, int32_t* F_out, void* cuda_stream)
{
    if (R < 1 || R > GL_STATIC_RMAX || m < 0 || m >= (1ll << 31) || !gamma || !loss_out || (m > 0 && !edges))
        return SB_ERR_ARG;
    // an error left pending by the caller's own earlier work is not ours to
    // clear; refuse to run rather than report it as this call's failure
    if (cudaPeekAtLastError() != cudaSuccess) return SB_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return SB_ERR_CUDA;
    }
    void* base = nullptr;
    {
        // first call on this device: look up the array's device address with
        // the device current (the host-side symbol is not a device address)
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_gl_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SB_ERR_CUDA;
            }
            g_static_ptr[dev] = p;
        }
        base = g_static_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* red = (double*)base;
    int32_t* Facc = (int32_t*)(red + (size_t)GL_STATIC_BLOCKS * GL_STATIC_RMAX);
    if (cudaMemsetAsync(Facc, 0, sizeof(int32_t) * (size_t)R, st) != cudaSuccess) {
        cudaGetLastError();
        return SB_ERR_CUDA;
    }
    k_gl_fwd<<<GL_STATIC_BLOCKS, GL_THREADS, 0, st>>>((const int2*)edges, m, gamma, R, red, Facc);
    if (cudaGetLastError() != cudaSuccess) return SB_ERR_CUDA;
    k_gl_fwd_final<<<(unsigned)sb_cdiv(R, 256), 256, 0, st>>>(red, GL_STATIC_BLOCKS, R, m, loss_out, Facc, F_out);
    if (cudaGetLastError() != cudaSuccess) return SB_ERR_CUDA;
    return SB_OK;
}
