// ubench.cu -- register-only throughput of the modular primitives the kernels are built
// from (Harvey lazy butterfly, 64x64->128 multiply-accumulate, Barrett product), used
// as the measured integer roofline of the ALU-bound kernels.  Each thread runs
// independent chains on register values; nothing touches memory except one store
// per thread at the end (so the work cannot be optimised away).
#include <algorithm>

#include "ntt_block.cuh"
#include "ops.cuh"

__global__ void ub_butterfly(u64 *sink, u64 q, u64 w, u64 ws, u32 iters) {
    u64 a0 = threadIdx.x + 1, a1 = blockIdx.x + 3, a2 = a0 * 7 + 5, a3 = a1 * 11 + 13;
    u64 b0 = a0 ^ 99, b1 = a1 ^ 77, b2 = a2 ^ 55, b3 = a3 ^ 33;
    const u64 q2 = 2 * q;
#define UB_BFLY(U, X)                       \
    {                                       \
        if (U >= q2) U -= q2;               \
        const u64 V = shoup_lazy(X, w, ws, q); \
        const u64 T = U + V;                \
        X = U - V + q2;                     \
        U = T;                              \
    }
    for (u32 i = 0; i < iters; ++i) {
        UB_BFLY(a0, b0);
        UB_BFLY(a1, b1);
        UB_BFLY(a2, b2);
        UB_BFLY(a3, b3);
    }
#undef UB_BFLY
    sink[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ b0 ^ b1 ^ b2 ^ b3;
}

__global__ void ub_mac128(u64 *sink, u64 x, u32 iters) {
    const u64 M61 = (1ull << 61) - 1;   // operands below 2^61 like the residues
    Acc128 acc[8];
    u64 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc[k].lo = acc[k].hi = 0;
        v[k] = (x * (threadIdx.x + 7 * k + 1)) & M61;
    }
    const u64 w = (x ^ 0x5bd1e995ull) & M61;
    for (u32 i = 0; i < iters; ++i) {
        const u64 y = (w + i) & M61;
#pragma unroll
        for (int k = 0; k < 8; ++k) mac128(acc[k], v[k], y);
    }
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= acc[k].lo ^ acc[k].hi;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ub_barrett(u64 *sink, PrimeDev P, u32 iters) {
    u64 a[4] = {threadIdx.x + 1ull, blockIdx.x + 2ull, threadIdx.x * 3ull + 7, blockIdx.x * 5ull + 9};
    const u64 b = P.q - 12345;
    for (u32 i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = mul_mod(a[k], b, P);
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = a[0] ^ a[1] ^ a[2] ^ a[3];
}

// Times each primitive with CUDA events on the context's stream; results per second:
// out[0] butterflies/s, out[1] 64x64->128 multiply-accumulates/s, out[2] Barrett products/s,
// out[3] the SM count the grids were sized for (SMs x resident CTAs per SM of each kernel).
extern "C" he_status he_ubench(he_ctx *h, double *out) {
    try {
        if (!h || !h->c || !out) return HE_EINVAL;
        Ctx *c = h->c.get();
        CtxLock lk(c);
        CUDA_TRY(cudaSetDevice(c->device));
        // every SM of this device filled to the occupancy each kernel reaches
        int sms = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
        const u32 threads = 256, iters = 4096;
        int occ[3] = {0, 0, 0};
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], ub_butterfly, threads, 0));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], ub_mac128, threads, 0));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], ub_barrett, threads, 0));
        u32 grid[3];
        for (int k = 0; k < 3; ++k) grid[k] = (u32)sms * (u32)std::max(1, occ[k]);
        const u32 blocks = std::max(grid[0], std::max(grid[1], grid[2]));
        DBuf sink(c, (size_t)blocks * threads);
        const PrimeDev P = c->pdev_h[0];
        const u64 w = P.q / 3, ws = (u64)(((unsigned __int128)w << 64) / P.q);
        cudaEvent_t e0, e1;
        CUDA_TRY(cudaEventCreate(&e0));
        CUDA_TRY(cudaEventCreate(&e1));
        float ms;
        const double nthr0 = (double)grid[0] * threads, nthr1 = (double)grid[1] * threads,
                     nthr2 = (double)grid[2] * threads;
        // a warm-up run, then the best of three timed runs of each
        out[0] = out[1] = out[2] = 0;
        out[3] = sms;
        for (int rep = 0; rep < 4; ++rep) {
            CUDA_TRY(cudaEventRecord(e0, c->stream));
            ub_butterfly<<<grid[0], threads, 0, c->stream>>>(sink.p, P.q, w, ws, iters);
            CUDA_TRY(cudaEventRecord(e1, c->stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep) out[0] = std::max(out[0], nthr0 * iters * 4 / (ms * 1e-3));
            CUDA_TRY(cudaEventRecord(e0, c->stream));
            ub_mac128<<<grid[1], threads, 0, c->stream>>>(sink.p, P.q - 1, iters);
            CUDA_TRY(cudaEventRecord(e1, c->stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep) out[1] = std::max(out[1], nthr1 * iters * 8 / (ms * 1e-3));
            CUDA_TRY(cudaEventRecord(e0, c->stream));
            ub_barrett<<<grid[2], threads, 0, c->stream>>>(sink.p, P, iters);
            CUDA_TRY(cudaEventRecord(e1, c->stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep) out[2] = std::max(out[2], nthr2 * iters * 4 / (ms * 1e-3));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->launches += 12;
        return HE_OK;
    } catch (const HeError &e) {
        return e.code;
    }
}
