// noalloc.cu -- a rescale entry point that performs no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// rescale: code running inside a CUDA stream capture (cudaMalloc is not a
// stream operation and breaks the capture), serving processes that reserve
// their whole memory budget up front and must never fail with out-of-memory
// in the middle of a request, and hosts whose device memory is entirely
// owned by another allocator (for example a framework's caching allocator).
// he_rescale_noalloc serves them: the caller passes input and output buffers,
// the context's tables were allocated when the context was created, and the
// only working memory -- the top limb of every polynomial in coefficient form
// -- lives in the file-scope device array below, which every GPU that loads
// the library holds until the process exits.
#include <mutex>

#include "ntt_block.cuh"
#include "ops.cuh"

// scratch: 2*batch rows of N words; 2^19 words (4 MiB) = batch <= 16 at N = 2^14
#define NOALLOC_SCRATCH_WORDS (1u << 19)
static __device__ __align__(256) u64 g_rescale_scratch[NOALLOC_SCRATCH_WORDS];

namespace {
struct RescaleConsts {
    u64 w[HE_MAX_PRIMES];    // q_top^{-1} mod q_i
    u64 ws[HE_MAX_PRIMES];   // Shoup companions
};

std::mutex g_mu;
u64 *g_addr[64];
bool g_ready[64];

// Device address of the scratch array for the current device.  In host code the
// name g_rescale_scratch is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and then reused.
u64 *scratch_address(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) throw HeError(HE_EINVAL, "device ordinal out of range");
    if (!g_ready[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rescale_scratch);
        if (e != cudaSuccess) throw HeError(HE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<u64 *>(p);
        g_ready[dev] = true;
    }
    return g_addr[dev];
}

u64 mulmod_n(u64 a, u64 b, u64 q) { return (u64)((unsigned __int128)a * b % q); }
u64 powmod_n(u64 a, u64 e, u64 q) {
    u64 r = 1;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_n(r, a, q);
        a = mulmod_n(a, a, q);
        e >>= 1;
    }
    return r;
}
}  // namespace

// scratch[r][n] = in[(r*lp + lp-1)*N + n]: the top limb of each of the 2*batch polynomials
__global__ void noalloc_gather_top(u64 *scratch, const u64 *__restrict__ in, u32 rows, u32 lp, u32 logn) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * N) return;
    size_t r = idx >> logn;
    scratch[idx] = in[(r * lp + lp - 1) * N + (idx & (N - 1))];
}

// inverse NTT of every scratch row (all rows use the top prime)
__global__ void __launch_bounds__(NTT_MAX_THREADS) noalloc_intt(u64 *scratch, u32 prime, const u64 *tw_all,
                                                                const PrimeDev *pd, int logn) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    u64 *g = scratch + (size_t)blockIdx.x * N;
    const PrimeDev P = pd[prime];
    block_load(sm, g, N);
    block_ntt_inv(sm, logn, tw_all + (size_t)prime * 4 * N, P.q, P.ninv, P.ninvs);
    block_store(g, sm, N);
}

// c'_i = (c_i - [c_top]_centred) * q_top^{-1} mod q_i, per (limb i, poly k, ciphertext b)
__global__ void __launch_bounds__(NTT_MAX_THREADS) noalloc_rescale(u64 *out, const u64 *__restrict__ in,
                                                                   const u64 *__restrict__ top, u32 lp, int logn,
                                                                   RescaleConsts rc, const u64 *__restrict__ tw_all,
                                                                   const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    const u32 i = blockIdx.x, k = blockIdx.y, b = blockIdx.z;
    const PrimeDev P = pd[i];
    const u64 qt = pd[lp - 1].q;
    const u64 *tb = top + ((size_t)b * 2 + k) * N;
    for (u32 n = threadIdx.x; n < N; n += blockDim.x) {
        u64 v = tb[n];
        sm[spad(n)] = v > qt / 2 ? neg_mod(reduce64(qt - v, P), P.q) : reduce64(v, P);
    }
    __syncthreads();
    block_ntt_fwd(sm, logn, tw_all + (size_t)i * 4 * N, P.q);
    const u64 *ib = in + (((size_t)b * 2 + k) * lp + i) * N;
    u64 *ob = out + (((size_t)b * 2 + k) * (lp - 1) + i) * N;
    for (u32 n = threadIdx.x; n < N; n += blockDim.x)
        ob[n] = mul_shoup(sub_mod(ib[n], sm[spad(n)], P.q), rc.w[i], rc.ws[i], P.q);
}

extern const char *set_last_error(const char *msg);

extern "C" he_status he_rescale_noalloc(he_ctx *h, const uint64_t *in, uint64_t *out, uint32_t batch,
                                        uint32_t limbs) {
    try {
        if (!h || !h->c) throw HeError(HE_EINVAL, "null context");
        Ctx *c = h->c.get();
        CtxLock lk(c);
        if (!in || !out || !batch) throw HeError(HE_EINVAL, "null buffer or empty batch");
        if (limbs < 2) throw HeError(HE_ELEVEL, "rescale needs at least two limbs");
        if (limbs > c->L1) throw HeError(HE_EINVAL, "more limbs than data primes");
        if (c->logn > 14) throw HeError(HE_EINVAL, "he_rescale_noalloc: N above 16384 is not supported");
        const u32 N = c->N;
        if ((size_t)batch * 2 * N > NOALLOC_SCRATCH_WORDS)
            throw HeError(HE_EINVAL, fmt("he_rescale_noalloc: batch*2*N = %zu words exceeds the %u-word scratch "
                                         "(at most %u ciphertexts at N = %u)",
                                         (size_t)batch * 2 * N, NOALLOC_SCRATCH_WORDS,
                                         NOALLOC_SCRATCH_WORDS / (2 * N), N));
        {
            // the kernels read `in` while other blocks write `out` (with another limb stride):
            // the two ranges must not share a word
            const uintptr_t i0 = (uintptr_t)in, i1 = i0 + (uintptr_t)batch * 2 * limbs * N * 8;
            const uintptr_t o0 = (uintptr_t)out, o1 = o0 + (uintptr_t)batch * 2 * (limbs - 1) * N * 8;
            if (i0 < o1 && o0 < i1) throw HeError(HE_EINVAL, "he_rescale_noalloc: in and out overlap");
        }
        CUDA_TRY(cudaSetDevice(c->device));
        u64 *scratch = scratch_address(c->device);
        static std::once_flag attr_once[64];
        std::call_once(attr_once[c->device & 63], [] {
            cudaFuncSetAttribute(noalloc_intt, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            cudaFuncSetAttribute(noalloc_rescale, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        });
        RescaleConsts rc;
        memset(&rc, 0, sizeof rc);
        const u64 qt = c->primes[limbs - 1];
        for (u32 i = 0; i + 1 < limbs; ++i) {
            const u64 qi = c->primes[i];
            rc.w[i] = powmod_n(qt % qi, qi - 2, qi);
            rc.ws[i] = (u64)(((unsigned __int128)rc.w[i] << 64) / qi);
        }
        const u32 rows = 2 * batch;
        const size_t total = (size_t)rows * N;
        const size_t smem = (size_t)ntt_smem_words(N) * 8;
        noalloc_gather_top<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(scratch, in, rows, limbs, c->logn);
        noalloc_intt<<<rows, ntt_threads(N), smem, c->stream>>>(scratch, limbs - 1, c->tw, c->pdev, c->logn);
        dim3 grid(limbs - 1, 2, batch);
        noalloc_rescale<<<grid, ntt_threads(N), smem, c->stream>>>(out, in, scratch, limbs, c->logn, rc, c->tw,
                                                                    c->pdev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) throw HeError(HE_ECUDA, std::string("he_rescale_noalloc: ") + cudaGetErrorString(e));
        c->launches += 3;
        return HE_OK;
    } catch (const HeError &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HE_EINVAL;
    }
}
