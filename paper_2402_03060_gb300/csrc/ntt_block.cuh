// ntt_block.cuh -- negacyclic NTT of one limb held in shared memory by a whole CTA.
//
// Forward: Cooley-Tukey butterflies with psi powers in bit-reversed order
// (Longa & Naehrig 2016, Alg. 1), output in bit-reversed evaluation order:
// slot i holds a(psi^(2*brev(i)+1)).  Inverse: Gentleman-Sande with inverse
// psi powers (their Alg. 2) followed by the N^{-1} scaling.  Twiddle tables
// per prime: [psi_rev | psi_rev_shoup | ipsi_rev | ipsi_rev_shoup], N words each.
//
// Lazy reduction (Harvey 2014): values are kept in [0, 4q) between the
// butterflies of the forward transform and in [0, 2q) in the inverse one, and
// reduced to [0, q) at the end; all primes are below 2^61, so 4q < 2^63.
#pragma once
#include "he_internal.cuh"

__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
    // a * w mod q in [0, 2q) for any a < 2^64
    u64 qh = mulhi64(a, ws);
    return a * w - qh * q;
}

// in-place forward transform of a[0..N) in shared memory; all threads of the CTA call it.
__device__ __forceinline__ void block_ntt_fwd(u64 *a, int logn, const u64 *__restrict__ tw, u64 q) {
    const u32 N = 1u << logn;
    const u64 *tws = tw + N;
    const u64 q2 = 2 * q, q4 = 4 * q;
    for (int lgm = 0; lgm < logn; ++lgm) {
        const int lgt = logn - 1 - lgm;
        const u32 t = 1u << lgt;
        for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const u32 i = b >> lgt;
            const u32 j = (i << (lgt + 1)) + (b & (t - 1));
            const u64 S = __ldg(tw + (1u << lgm) + i);
            const u64 Ss = __ldg(tws + (1u << lgm) + i);
            u64 U = a[j];
            if (U >= q2) U -= q2;
            const u64 V = shoup_lazy(a[j + t], S, Ss, q);
            a[j] = U + V;                 // < 4q
            a[j + t] = U - V + q2;        // < 4q
        }
        __syncthreads();
    }
    for (u32 k = threadIdx.x; k < N; k += blockDim.x) {
        u64 v = a[k];
        if (v >= q2) v -= q2;
        if (v >= q) v -= q;
        a[k] = v;
    }
    __syncthreads();
}

// in-place inverse transform including the N^{-1} factor; input in [0, q).
__device__ __forceinline__ void block_ntt_inv(u64 *a, int logn, const u64 *__restrict__ tw, u64 q, u64 ninv,
                                              u64 ninvs) {
    const u32 N = 1u << logn;
    const u64 *itw = tw + 2 * N;
    const u64 *itws = tw + 3 * N;
    const u64 q2 = 2 * q;
    for (int lgt = 0; lgt < logn; ++lgt) {
        const u32 t = 1u << lgt;
        const u32 h = N >> (lgt + 1);
        for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const u32 i = b >> lgt;
            const u32 j = (i << (lgt + 1)) + (b & (t - 1));
            const u64 S = __ldg(itw + h + i);
            const u64 Ss = __ldg(itws + h + i);
            const u64 U = a[j], V = a[j + t];   // both < 2q
            u64 s = U + V;
            if (s >= q2) s -= q2;
            a[j] = s;                          // < 2q
            a[j + t] = shoup_lazy(U - V + q2, S, Ss, q);   // < 2q
        }
        __syncthreads();
    }
    for (u32 k = threadIdx.x; k < N; k += blockDim.x) a[k] = mul_shoup(a[k], ninv, ninvs, q);
    __syncthreads();
}

__device__ __forceinline__ void block_load(u64 *s, const u64 *__restrict__ g, u32 N) {
    const ulonglong2 *g2 = reinterpret_cast<const ulonglong2 *>(g);
    ulonglong2 *s2 = reinterpret_cast<ulonglong2 *>(s);
    for (u32 k = threadIdx.x; k < N / 2; k += blockDim.x) s2[k] = g2[k];
    __syncthreads();
}
__device__ __forceinline__ void block_store(u64 *__restrict__ g, const u64 *s, u32 N) {
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(s);
    ulonglong2 *g2 = reinterpret_cast<ulonglong2 *>(g);
    for (u32 k = threadIdx.x; k < N / 2; k += blockDim.x) g2[k] = s2[k];
}

static inline u32 ntt_threads(u32 N) { return N >= 2048 ? 1024 : N / 2; }
