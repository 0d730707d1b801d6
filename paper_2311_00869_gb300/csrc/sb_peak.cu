// sb_peak.cu -- measured integer-ALU ceiling of the BFS parent-key hash.
//
// The randomized BFS (Algorithm 1's tree sampler) spends its time hashing
// parent candidates: per candidate (tree t, neighbour u, vertex v) it adds the
// tree salt to u ^ y_v (computed once per neighbour), applies the 32-bit
// MurmurHash3 finaliser and keeps the running minimum.  k_hash_peak runs
// exactly that mix -- one add, sb_fmix32, one min -- on independent chains in
// every thread of a full grid, with nothing else in the loop, so its rate is
// the ceiling the BFS's hash work can reach on this GPU.
#include <algorithm>

#include "sb_internal.cuh"

#define PK_THREADS 256
#define PK_CHAINS 8  // independent hash chains per thread (instruction-level parallelism)

__global__ void __launch_bounds__(PK_THREADS) k_hash_peak(int iters, uint32_t salt0, uint32_t step,
                                                          uint32_t* __restrict__ sink)
{
    const uint32_t tid = blockIdx.x * PK_THREADS + threadIdx.x;
    uint32_t x[PK_CHAINS], best[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) {
        x[k] = sb_fmix32(tid * PK_CHAINS + k + 1u);  // u ^ y_v of one candidate neighbour
        best[k] = 0xFFFFFFFFu;
    }
    uint32_t a = salt0;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) best[k] = min(best[k], sb_fmix32(x[k] + a));
        a += step;  // the next tree's salt
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) r ^= best[k];
    if (r == 0x5EED5EEDu) sink[0] = r;  // keeps the chains alive; practically never taken
}

extern "C" sb_status sb_hash_peak(sb_ctx* c, double seconds, double* hashes_per_s_out)
{
    if (!c || !hashes_per_s_out || !(seconds > 0.0) || seconds > 60.0) return SB_ERR_ARG;
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_ensure(c, &c->tmp, &c->tmp_cap, 256));
    int per_sm = 0;
    SB_CHECK_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hash_peak, PK_THREADS, 0));
    if (per_sm < 1) return sb_fail(c, SB_ERR_CUDA, "hash peak kernel does not fit on an SM");
    const unsigned blocks = (unsigned)(per_sm * c->num_sms);
    cudaEvent_t e0, e1;
    SB_CHECK_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return sb_cuda_fail(c, cudaGetLastError(), "cudaEventCreate");
    }
    auto run = [&](int iters, float* ms) -> cudaError_t {
        cudaEventRecord(e0, c->stream);
        k_hash_peak<<<blocks, PK_THREADS, 0, c->stream>>>(iters, 0x243F6A88u, 0x632BE5ABu, (uint32_t*)c->tmp);
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        return e;
    };
    // warm up and calibrate on a short run, then time one run of `seconds`
    int iters = 1 << 12;
    float ms = 0.f;
    cudaError_t err = run(iters, &ms);
    for (int k = 0; k < 3 && err == cudaSuccess; k++) {
        const double want = seconds * 1000.0;
        const double scale = ms > 0.01f ? want / ms : 16.0;
        const double next = (double)iters * (k < 2 ? std::min(scale, 16.0) : scale);
        iters = (int)std::max(1.0, std::min(next, 2.0e9));
        err = run(iters, &ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return sb_cuda_fail(c, err, "k_hash_peak");
    const double hashes = (double)blocks * PK_THREADS * PK_CHAINS * (double)iters;
    *hashes_per_s_out = hashes / (ms / 1000.0);
    return SB_OK;
}
