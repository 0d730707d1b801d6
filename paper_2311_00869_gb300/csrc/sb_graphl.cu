// sb_graphl.cu -- graphL (Sec. 4, Alg. 2): relaxed loss (Eq. 3), discrete
// loss (Eq. 2), the adjoint dL/dG_v = -1/2 sum_j e_vj G_j (Eq. 4), the descent
// update G <- G - alpha dL/dG, and the final rounding (Alg. 2 lines 11-24).
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

struct GlArgs {
    const sb_bfs_item* items;
    int64_t n_items;
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* hub_first;
    const float* gin;      // n x R input
    float* gout_rows;      // n x R output
    float* partial;        // partial sums of split rows
    const float* upstream; // GRAD: gout[R]
    const float* scale;    // STEP: per-column input scale (power of two)
    float half_alpha;      // STEP: alpha / 2
    int32_t* F;            // STEP: per-column discrete-loss accumulator (x2), nullable
    uint32_t* colmax;      // STEP: per-column max |G_out| bits
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

// epilogue shared by whole rows and by combined split rows
template <bool STEP>
__device__ __forceinline__ void gl_emit(const GlArgs& A, int64_t v, int r, float acc, int32_t* sF, uint32_t* smax)
{
    const int64_t idx = v * A.R + r;
    if (!STEP) {
        A.gout_rows[idx] = -0.5f * A.upstream[r] * acc;
    } else {
        const float sc = A.scale[r];
        const float g = A.gin[idx] * sc;
        const float out = g + A.half_alpha * (acc * sc);
        A.gout_rows[idx] = out;
        atomicMax(smax + r, __float_as_uint(fabsf(out)));
    }
}

// Rows (and chunks of split rows): a sub-warp of SL lanes per (item, segment
// of SL*VEC columns).  Units run segment-major, so one segment's columns of G
// (n x SL*VEC floats; 84 MB for 656k vertices at 32 columns) stay in L2 while
// every row gathers from them.
template <int VEC, int SL, bool STEP>
__global__ void __launch_bounds__(GL_THREADS) k_gl_rows(GlArgs A)
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
    const int64_t units = A.n_items * nseg;
    const bool wantF = STEP && A.F != nullptr;
    for (int64_t u = sub_id; u < units; u += subs_total) {
        const int seg = (int)(u / A.n_items);
        const int64_t it = u - (int64_t)seg * A.n_items;
        const sb_bfs_item itm = A.items[it];
        const int r0 = seg * seg_w + sl * VEC;
        const bool act = r0 < R;
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
                for (int q = 0; q < cc_n; q++) {
                    const uint32_t cc = __shfl_sync(smask, mycol, q, SL);
                    const uint32_t nb = cc & 0x80000000u;
                    const uint32_t nb1 = cc >> 31;
                    const int64_t base = (int64_t)(cc & SB_ID_MASK) * R + r0;
                    if (act) {
                        if (VEC == 4) {
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
            for (int k = 0; k < VEC; k++)
                if (r0 + k < R && fcnt[k]) atomicAdd(sF + r0 + k, fcnt[k]);
        }
        if (itm.hub >= 0) {
            const int64_t slot = A.hub_first[itm.hub] + (itm.beg - A.rowptr[itm.v]) / SB_GL_CHUNK;
#pragma unroll
            for (int k = 0; k < VEC; k++)
                if (r0 + k < R) A.partial[slot * R + r0 + k] = acc[k];
        } else {
#pragma unroll
            for (int k = 0; k < VEC; k++)
                if (r0 + k < R) gl_emit<STEP>(A, itm.v, r0 + k, acc[k], sF, smax);
        }
    }
    if (STEP) {
        __syncthreads();
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
    int32_t* sF = (int32_t*)gsm;
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
        gl_emit<STEP>(A, hub_vertex[h], r, acc, sF, smax);
    }
    if (STEP) {
        __syncthreads();
        for (int i = threadIdx.x; i < R; i += GL_THREADS)
            if (smax[i]) atomicMax(A.colmax + i, smax[i]);
    }
}

// per-column renorm decision and discrete-loss trace after one step
__global__ void k_gl_step_final(int R, uint32_t* colmax, int32_t* Facc, int32_t* F_trace_row, float* scale,
                                int32_t* exps, int renorm_log2)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
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

__global__ void k_gl_fill(float* p, int R, float v)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) p[r] = v;
}

__global__ void k_gl_apply_scale(float* g, int64_t n, int R, const float* scale)
{
    const int64_t total = n * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        g[i] *= scale[i % R];
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
                                                         uint64_t* flips)
{
    const int64_t nw = sb_cdiv(m, 64);
    for (int64_t w = blockIdx.x; w < nw; w += gridDim.x) {
        const int64_t e0 = w * 64;
        const int cnt = (int)min((int64_t)64, m - e0);
        for (int r = threadIdx.x; r < R; r += GL_THREADS) {
            uint64_t bits = 0;
            for (int k = 0; k < cnt; k++) {
                const int2 ed = edges[e0 + k];
                const uint32_t a = is_neg(g[(int64_t)ed.x * R + r]);
                const uint32_t b = is_neg(g[(int64_t)((uint32_t)ed.y & SB_ID_MASK) * R + r]);
                bits |= (uint64_t)(a ^ b ^ ((uint32_t)ed.y >> 31)) << k;
            }
            if (flips) flips[(int64_t)r * nw + w] = bits;
            const int c = __popcll(bits);
            if (c) atomicAdd(Facc + r, c);
        }
    }
}

__global__ void k_gl_copy_F(int32_t* Facc, int R, int32_t* out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
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
    SB_TRY(sb_ensure(c, (void**)&c->gl_misc, &c->gl_misc_cap, sizeof(int32_t) * (size_t)4 * R + 64));
    if (need_buf) SB_TRY(sb_ensure(c, (void**)&c->gl_buf, &c->gl_buf_cap, sizeof(float) * (size_t)c->n * R));
    return SB_OK;
}

static GlArgs gl_args(sb_ctx* c, int R)
{
    GlArgs A;
    memset(&A, 0, sizeof(A));
    A.items = c->gl_items;
    A.n_items = c->n_gl_items;
    A.rowptr = c->rowptr;
    A.col = c->col;
    A.hub_first = c->gl_hub_first;
    A.partial = c->gl_partial;
    A.n = c->n;
    A.R = R;
    return A;
}

template <bool STEP>
static sb_status gl_rows_launch(sb_ctx* c, GlArgs& A)
{
    const bool vec4 = (A.R % 4 == 0) && (((uintptr_t)A.gin & 15) == 0);
    const void* fn = vec4 ? (const void*)k_gl_rows<4, 8, STEP> : (const void*)k_gl_rows<1, 32, STEP>;
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
    int32_t* Facc = c->gl_misc;
    SB_CHECK_CUDA(c, cudaMemsetAsync(Facc, 0, sizeof(int32_t) * R, c->stream));
    unsigned blocks = (unsigned)std::min<int64_t>(std::max<int64_t>(sb_cdiv(c->m, 64), 1), (int64_t)c->num_sms * 8);
    SbProf prof(c, SB_PROF_GL_FWD);
    k_gl_round<<<blocks, GL_THREADS, 0, c->stream>>>(c->edges, c->m, gamma, R, Facc, flip_out);
    SB_TRY(sb_after_launch(c, "k_gl_round"));
    k_gl_copy_F<<<(unsigned)sb_cdiv(R, 256), 256, 0, c->stream>>>(Facc, R, F_out);
    return sb_after_launch(c, "k_gl_copy_F");
}

extern "C" sb_status sb_graphL_descent(sb_ctx* c, const float* gamma0, float* gamma_out, int32_t R, float alpha,
                                       int32_t steps, int32_t renorm_log2, int32_t* exps_out, int32_t* F_trace,
                                       int32_t* F_final)
{
    SB_TRY(gl_check(c, R));
    if (!gamma0 || !gamma_out || !exps_out || steps < 0 || renorm_log2 < 0 || renorm_log2 > 100)
        return sb_fail(c, SB_ERR_ARG, "bad descent argument");
    SB_TRY(gl_scratch(c, R, true));
    if (!c->gl_scale) c->gl_scale = (float*)sb_dalloc(c, sizeof(float) * 65536);
    if (!c->gl_colmax) c->gl_colmax = (uint32_t*)sb_dalloc(c, sizeof(uint32_t) * 65536);
    if (!c->gl_scale || !c->gl_colmax) return sb_fail(c, SB_ERR_OOM, "descent scratch");
    const size_t bytes = sizeof(float) * (size_t)c->n * R;
    int32_t* Facc = c->gl_misc;
    SB_CHECK_CUDA(c, cudaMemsetAsync(Facc, 0, sizeof(int32_t) * R, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->gl_colmax, 0, sizeof(uint32_t) * R, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(exps_out, 0, sizeof(int32_t) * R, c->stream));
    unsigned rb = (unsigned)sb_cdiv(R, 256);
    k_gl_fill<<<rb, 256, 0, c->stream>>>(c->gl_scale, R, 1.0f);
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
    for (int s = 0; s < steps; s++) {
        float* dst = (src == gamma_out) ? c->gl_buf : gamma_out;
        A.gin = src;
        A.gout_rows = dst;
        A.F = F_trace ? Facc : nullptr;
        SB_TRY(gl_rows_launch<true>(c, A));
        k_gl_step_final<<<rb, 256, 0, c->stream>>>(R, c->gl_colmax, Facc, F_trace ? F_trace + (int64_t)s * R : nullptr,
                                                   c->gl_scale, exps_out, renorm_log2);
        SB_TRY(sb_after_launch(c, "k_gl_step_final"));
        src = dst;
    }
    if (src != gamma_out) SB_CHECK_CUDA(c, cudaMemcpyAsync(gamma_out, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    // pending power-of-two scale of the last step
    unsigned gb = (unsigned)std::min<int64_t>(sb_cdiv((int64_t)c->n * R, 256), (int64_t)c->num_sms * 16);
    k_gl_apply_scale<<<gb, 256, 0, c->stream>>>(gamma_out, c->n, R, c->gl_scale);
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
    k_gl_fwd_final<<<(unsigned)sb_cdiv(R, 256), 256, 0, st>>>(red, GL_STATIC_BLOCKS, R, m, loss_out, Facc, F_out);
    if (cudaGetLastError() != cudaSuccess) return SB_ERR_CUDA;
    return SB_OK;
}
