// ntt_block.cuh -- negacyclic NTT of one limb held in shared memory by a whole CTA.
//
// Forward: Cooley-Tukey butterflies with psi powers in bit-reversed order
// (Longa & Naehrig 2016, Alg. 1), output in bit-reversed evaluation order:
// slot i holds a(psi^(2*brev(i)+1)).  Inverse: Gentleman-Sande with inverse
// psi powers (their Alg. 2) followed by the N^{-1} scaling.  Twiddle table per
// prime (4N words): N pairs (psi_rev[i], Shoup companion), then N pairs for the
// inverse powers -- one 16-byte load per twiddle.
//
// Lazy reduction (Harvey 2014): values stay in [0, 4q) between forward
// butterflies and in [0, 2q) between inverse ones; all primes are below 2^61.
//
// Register blocking: for N >= 1024 every thread holds 16 coefficients of a
// butterfly group and runs 4 stages on them in registers, so a limb of 2^14
// coefficients takes 4 shared-memory passes (and 4 barriers) instead of 14,
// and a group loads 15 twiddle pairs for 32 butterflies.  Shared memory is
// padded by one word per 16 so that the strided group loads are conflict-free.
//
// The two-kernel form at the end of this file transforms a limb by two launches instead
// (outer stages over columns in registers, inner stages over 1024-coefficient blocks).
//
// Limbs larger than one CTA's shared memory (N = 2^15: 256 KiB) are split over
// a cluster of two CTAs ("parts"): CTA r holds coefficients [r*N/2, (r+1)*N/2).
// The one stage whose butterflies join the halves (distance N/2: the first
// forward stage, the last inverse one) reads and writes the peer's half through
// distributed shared memory; every other stage is local, with the twiddle index
// taken from the global coefficient index.
#pragma once
#include <cooperative_groups.h>

#include "he_internal.cuh"

__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
    // a * w mod q in [0, 2q) for any a < 2^64
    u64 qh = mulhi64(a, ws);
    return a * w - qh * q;
}

__device__ __forceinline__ u32 spad(u32 i) { return i + (i >> 4); }
// shared-memory words a limb of N coefficients occupies (padded)
__host__ __device__ __forceinline__ u32 ntt_smem_words(u32 N) { return N + N / 16; }

// threads of a CTA that transforms one limb: two 16-coefficient register groups
// per thread per pass (so a thread may use up to 128 registers without spilling)
#define NTT_MAX_THREADS 512
static inline u32 ntt_threads(u32 N) { return N >= 1024 ? N / 32 : (N / 2 < 32 ? 32 : N / 2); }

// largest limb one CTA transforms alone; above it a limb must be split over a
// 2-CTA cluster (below it splitting is a tuning choice: half the shared memory
// and threads per CTA, more CTAs resident per SM, one DSMEM exchange stage)
#define NTT_PART_LOGN 14
static inline int ntt_min_split(int logn) { return logn > NTT_PART_LOGN ? 1 : 0; }
static inline int ntt_can_split(int logn) { return logn >= 11; }
// coefficients one CTA holds, its threads and its dynamic shared memory
static inline u32 ntt_part_n(int logn, int split) { return 1u << (logn - split); }
static inline u32 ntt_part_threads(int logn, int split) { return ntt_threads(ntt_part_n(logn, split)); }
static inline size_t ntt_part_smem(int logn, int split) { return (size_t)ntt_smem_words(ntt_part_n(logn, split)) * 8; }

// which part of the limb this CTA holds: coefficients [lo, lo + n).  Kernels
// are instantiated for SPLIT = 0 (one CTA per limb) and SPLIT = 1 (clusters of
// two CTAs along x, each limb split over the pair).
struct Part {
    u32 lo, n;
    int split;
};
template <int SPLIT>
__device__ __forceinline__ Part ntt_part(int logn) {
    Part p;
    p.split = SPLIT;
    p.n = 1u << (logn - SPLIT);
    p.lo = SPLIT ? (blockIdx.x & 1u) * p.n : 0u;
    return p;
}
// limb-level grid index (blockIdx.x with the cluster rank removed)
template <int SPLIT>
__device__ __forceinline__ u32 part_row() { return blockIdx.x >> SPLIT; }

// launch kern0 (one CTA per limb) or kern1 (a cluster of two CTAs per limb along x);
// grid.x counts limbs
template <typename... KArgs, typename... Args>
static void launch_parts(Ctx *c, void (*kern0)(KArgs...), void (*kern1)(KArgs...), dim3 grid, int split,
                         u32 threads, size_t smem, Args... args) {
    if (!split) {
        kern0<<<grid, threads, smem, c->stream>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid.x * 2, grid.y, grid.z);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CUDA_TRY(cudaLaunchKernelEx(&cfg, kern1, args...));
}

// twiddle pair i of the forward / inverse table
__device__ __forceinline__ ulonglong2 tw_fwd(const u64 *__restrict__ tw, u32 i) {
    return __ldg(reinterpret_cast<const ulonglong2 *>(tw) + i);
}
__device__ __forceinline__ ulonglong2 tw_inv(const u64 *__restrict__ tw, u32 N, u32 i) {
    return __ldg(reinterpret_cast<const ulonglong2 *>(tw + 2 * (size_t)N) + i);
}

// ---------------------------------------------------------------- forward
__device__ __forceinline__ void fwd_radix2_stage(u64 *a, int logn, int lgm, const u64 *__restrict__ tw, u64 q) {
    const u32 N = 1u << logn;
    const u64 q2 = 2 * q;
    const int lgt = logn - 1 - lgm;
    const u32 t = 1u << lgt;
    for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
        const u32 i = b >> lgt;
        const u32 j = (i << (lgt + 1)) + (b & (t - 1));
        const ulonglong2 W = tw_fwd(tw, (1u << lgm) + i);
        const u64 S = W.x, Ss = W.y;
        u64 U = a[spad(j)];
        if (U >= q2) U -= q2;
        const u64 V = shoup_lazy(a[spad(j + t)], S, Ss, q);
        a[spad(j)] = U + V;
        a[spad(j + t)] = U - V + q2;
    }
}

// R stages starting at stage st on groups of 2^R coefficients held in registers.
// a holds the 2^logl coefficients starting at global index goff of an N = 2^logn
// limb; every butterfly group of these stages lies inside it.
// With LAST the outputs are reduced to [0, q) before they are stored.
template <int R, bool LAST = false>
__device__ __forceinline__ void fwd_pass(u64 *a, int logn, int st, const u64 *__restrict__ tw, u64 q,
                                         int logl, u32 goff) {
    const u64 q2 = 2 * q;
    const int lgt0 = logn - 1 - st;          // log2 of the first distance t0
    const int lgtl = lgt0 - (R - 1);         // log2 of the smallest distance
    const u32 tl = 1u << lgtl;
    const u32 groups = (1u << logl) >> R;
    for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
        const u32 base = ((g >> lgtl) << (lgt0 + 1)) + (g & (tl - 1));
        u64 v[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) v[k] = a[spad(base + ((u32)k << lgtl))];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int lgd = lgt0 - u;                 // distance 2^lgd at stage st+u
            const u32 m = 1u << (st + u);
            const int half = 1 << (R - 1 - u);
#pragma unroll
            for (int blk = 0; blk < (1 << u); ++blk) {
                const u32 j = goff + base + ((u32)(blk * 2 * half) << lgtl);
                const u32 i = j >> (lgd + 1);
                const ulonglong2 W = tw_fwd(tw, m + i);
                const u64 S = W.x, Ss = W.y;
#pragma unroll
                for (int h = 0; h < half; ++h) {
                    const int k = blk * 2 * half + h;
                    u64 U = v[k];
                    if (U >= q2) U -= q2;
                    const u64 V = shoup_lazy(v[k + half], S, Ss, q);
                    v[k] = U + V;
                    v[k + half] = U - V + q2;
                }
            }
        }
        if (LAST) {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) {
                u64 w = v[k];
                if (w >= q2) w -= q2;
                if (w >= q) w -= q;
                v[k] = w;
            }
        }
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) a[spad(base + ((u32)k << lgtl))] = v[k];
    }
}

// stages st0.. of the forward transform on the local coefficients, then the
// final reduction to [0, q)
__device__ __forceinline__ void fwd_local(u64 *a, int logn, int st0, const u64 *__restrict__ tw, u64 q, int logl,
                                          u32 goff) {
    const u32 L = 1u << logl;
    if (logn >= 10) {
        // the short pass ((logn - st0) mod 4 stages) first, on the largest distances, then
        // passes of four; the last one also reduces to [0, q)
        const int rem = (logn - st0) % 4;
        if (rem == 3) fwd_pass<3>(a, logn, st0, tw, q, logl, goff);
        if (rem == 2) fwd_pass<2>(a, logn, st0, tw, q, logl, goff);
        if (rem == 1) fwd_pass<1>(a, logn, st0, tw, q, logl, goff);
        if (rem) __syncthreads();
        int st = st0 + rem;
        for (; st + 4 < logn; st += 4) {
            fwd_pass<4>(a, logn, st, tw, q, logl, goff);
            __syncthreads();
        }
        fwd_pass<4, true>(a, logn, st, tw, q, logl, goff);
        __syncthreads();
        return;
    }
    for (int lgm = st0; lgm < logn; ++lgm) {
        fwd_radix2_stage(a, logn, lgm, tw, q);
        __syncthreads();
    }
    const u64 q2 = 2 * q;
    for (u32 k = threadIdx.x; k < L; k += blockDim.x) {
        u64 v = a[spad(k)];
        if (v >= q2) v -= q2;
        if (v >= q) v -= q;
        a[spad(k)] = v;
    }
    __syncthreads();
}

// in-place forward transform of a[spad(0..N)] in shared memory; output in [0, q).
__device__ __forceinline__ void block_ntt_fwd(u64 *a, int logn, const u64 *__restrict__ tw, u64 q) {
    fwd_local(a, logn, 0, tw, q, logn, 0);
}

// forward transform of the limb held by this CTA's part (the whole limb, or
// half of it in each CTA of a 2-CTA cluster).  Every CTA of the cluster calls it
// after writing its part; the output stays in the part's own shared memory.
__device__ __forceinline__ void part_ntt_fwd(u64 *a, const Part &p, int logn, const u64 *__restrict__ tw, u64 q) {
    if (!p.split) {
        block_ntt_fwd(a, logn, tw, q);
        return;
    }
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();  // both halves written
    u64 *a0 = cl.map_shared_rank(a, 0), *a1 = cl.map_shared_rank(a, 1);
    const u32 N = 1u << logn, H = p.n;
    const ulonglong2 W = tw_fwd(tw, 1);
    const u64 S = W.x, Ss = W.y, q2 = 2 * q;
    (void)N;
    // stage 0 (distance N/2): pairs (j, j + N/2) sit at local index j of CTA 0 and CTA 1;
    // each CTA takes half of the pairs
    const u32 j0 = p.lo / 2;
    for (u32 j = j0 + threadIdx.x; j < j0 + H / 2; j += blockDim.x) {
        u64 U = a0[spad(j)];
        if (U >= q2) U -= q2;
        const u64 V = shoup_lazy(a1[spad(j)], S, Ss, q);
        a0[spad(j)] = U + V;
        a1[spad(j)] = U - V + q2;
    }
    cl.sync();  // remote writes visible; no remote access after this point
    fwd_local(a, logn, 1, tw, q, logn - 1, p.lo);
}

// ---------------------------------------------------------------- inverse
__device__ __forceinline__ void inv_radix2_stage(u64 *a, int logn, int lgt, const u64 *__restrict__ tw, u64 q) {
    const u32 N = 1u << logn;
    const u64 q2 = 2 * q;
    const u32 t = 1u << lgt;
    const u32 h = N >> (lgt + 1);
    for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
        const u32 i = b >> lgt;
        const u32 j = (i << (lgt + 1)) + (b & (t - 1));
        const ulonglong2 W = tw_inv(tw, N, h + i);
        const u64 S = W.x, Ss = W.y;
        const u64 U = a[spad(j)], V = a[spad(j + t)];
        u64 s = U + V;
        if (s >= q2) s -= q2;
        a[spad(j)] = s;
        a[spad(j + t)] = shoup_lazy(U - V + q2, S, Ss, q);
    }
}

// R Gentleman-Sande stages with distances 2^lgtl .. 2^(lgtl+R-1) on the 2^logl
// coefficients starting at global index goff
// With LAST the outputs are multiplied by N^{-1} (ninv, Shoup companion ninvs) before they are stored.
template <int R, bool LAST = false>
__device__ __forceinline__ void inv_pass(u64 *a, int logn, int lgtl, const u64 *__restrict__ tw, u64 q, int logl,
                                         u32 goff, u64 ninv = 0, u64 ninvs = 0) {
    const u32 N = 1u << logn;
    const u64 q2 = 2 * q;
    const u32 tl = 1u << lgtl;
    const u32 groups = (1u << logl) >> R;
    for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
        const u32 base = ((g >> lgtl) << (lgtl + R)) + (g & (tl - 1));
        u64 v[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) v[k] = a[spad(base + ((u32)k << lgtl))];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int lgd = lgtl + u;               // distance at this stage
            const u32 h = N >> (lgd + 1);
            const int half = 1 << u;
#pragma unroll
            for (int blk = 0; blk < (1 << (R - 1 - u)); ++blk) {
                const u32 j = goff + base + ((u32)(blk * 2 * half) << lgtl);
                const u32 i = j >> (lgd + 1);
                const ulonglong2 W = tw_inv(tw, N, h + i);
                const u64 S = W.x, Ss = W.y;
#pragma unroll
                for (int hh = 0; hh < half; ++hh) {
                    const int k = blk * 2 * half + hh;
                    const u64 U = v[k], V = v[k + half];
                    u64 s = U + V;
                    if (s >= q2) s -= q2;
                    v[k] = s;
                    v[k + half] = shoup_lazy(U - V + q2, S, Ss, q);
                }
            }
        }
        if (LAST) {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) v[k] = mul_shoup(v[k], ninv, ninvs, q);
        }
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) a[spad(base + ((u32)k << lgtl))] = v[k];
    }
}

// inverse stages with distances 1 .. 2^(nst-1) on the local coefficients; with
// scale the last pass also multiplies by N^{-1} (the radix-2 path for N < 1024
// does it in a separate loop)
__device__ __forceinline__ void inv_local(u64 *a, int logn, int nst, const u64 *__restrict__ tw, u64 q, int logl,
                                          u32 goff, bool scale, u64 ninv, u64 ninvs) {
    if (logn >= 10) {
        // the short pass (nst mod 4 stages) first, on the smallest distances, then passes of
        // four; the last one also applies N^{-1} when asked
        const int rem = nst % 4;
        if (rem == 3) inv_pass<3>(a, logn, 0, tw, q, logl, goff);
        if (rem == 2) inv_pass<2>(a, logn, 0, tw, q, logl, goff);
        if (rem == 1) inv_pass<1>(a, logn, 0, tw, q, logl, goff);
        if (rem) __syncthreads();
        int lgt = rem;
        for (; lgt + 4 < nst; lgt += 4) {
            inv_pass<4>(a, logn, lgt, tw, q, logl, goff);
            __syncthreads();
        }
        if (scale)
            inv_pass<4, true>(a, logn, lgt, tw, q, logl, goff, ninv, ninvs);
        else
            inv_pass<4>(a, logn, lgt, tw, q, logl, goff);
        __syncthreads();
        return;
    }
    for (int lgt = 0; lgt < nst; ++lgt) {
        inv_radix2_stage(a, logn, lgt, tw, q);
        __syncthreads();
    }
    if (scale) {
        for (u32 k = threadIdx.x; k < (1u << logl); k += blockDim.x) a[spad(k)] = mul_shoup(a[spad(k)], ninv, ninvs, q);
        __syncthreads();
    }
}

// in-place inverse transform including the N^{-1} factor; input in [0, q).
__device__ __forceinline__ void block_ntt_inv(u64 *a, int logn, const u64 *__restrict__ tw, u64 q, u64 ninv,
                                              u64 ninvs) {
    inv_local(a, logn, logn, tw, q, logn, 0, true, ninv, ninvs);
}

// inverse transform of the limb held by this CTA's part (see part_ntt_fwd)
__device__ __forceinline__ void part_ntt_inv(u64 *a, const Part &p, int logn, const u64 *__restrict__ tw, u64 q,
                                             u64 ninv, u64 ninvs) {
    if (!p.split) {
        block_ntt_inv(a, logn, tw, q, ninv, ninvs);
        return;
    }
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    inv_local(a, logn, logn - 1, tw, q, logn - 1, p.lo, false, 0, 0);
    cl.sync();  // both halves through their local stages
    u64 *a0 = cl.map_shared_rank(a, 0), *a1 = cl.map_shared_rank(a, 1);
    const u32 N = 1u << logn, H = p.n;
    const ulonglong2 W = tw_inv(tw, N, 1);
    const u64 S = W.x, Ss = W.y, q2 = 2 * q;
    // last stage (distance N/2) fused with the N^{-1} factor
    const u32 j0 = p.lo / 2;
    for (u32 j = j0 + threadIdx.x; j < j0 + H / 2; j += blockDim.x) {
        const u64 U = a0[spad(j)], V = a1[spad(j)];
        u64 s = U + V;
        if (s >= q2) s -= q2;
        a0[spad(j)] = mul_shoup(s, ninv, ninvs, q);
        a1[spad(j)] = mul_shoup(shoup_lazy(U - V + q2, S, Ss, q), ninv, ninvs, q);
    }
    cl.sync();
}

// global <-> padded shared memory, 16-byte vector accesses on the global side
__device__ __forceinline__ void block_load(u64 *s, const u64 *__restrict__ g, u32 N) {
    const ulonglong2 *g2 = reinterpret_cast<const ulonglong2 *>(g);
    for (u32 k = threadIdx.x; k < N / 2; k += blockDim.x) {
        ulonglong2 v = g2[k];
        s[spad(2 * k)] = v.x;
        s[spad(2 * k + 1)] = v.y;
    }
    __syncthreads();
}
__device__ __forceinline__ void block_store(u64 *__restrict__ g, const u64 *s, u32 N) {
    ulonglong2 *g2 = reinterpret_cast<ulonglong2 *>(g);
    for (u32 k = threadIdx.x; k < N / 2; k += blockDim.x) {
        ulonglong2 v;
        v.x = s[spad(2 * k)];
        v.y = s[spad(2 * k + 1)];
        g2[k] = v;
    }
}

// ---------------------------------------------------------------- two-kernel form
// A limb of N = 2^logn (11 <= logn <= 15) transformed by two launches instead of one CTA (or
// cluster) holding it whole.  Write a coefficient index as j = 1024 k + e: the R = logn - 10
// "outer" stages (distances N/2 .. 1024) act on the 1024 columns {e + 1024 k : k < 2^R}, one
// column per thread in registers; the ten "inner" stages (distances 512 .. 1) act on each
// 1024-coefficient block alone, one small CTA per block with the block in shared memory.
// Forward: outer launch, then inner; inverse: inner, then outer (with the N^-1 factor).  Every
// butterfly is the one-CTA transform's (same twiddle, same lazy reduction), so the results are
// the same bits.  The blocks are independent, so many small CTAs share an SM and their loads,
// stores and arithmetic overlap -- the one-CTA form runs one 512-thread CTA per SM at N = 2^14
// with all its warps in the same phase.  Cost: one more pass of the limb through L2 / HBM.
#define NTT2_INNER_LOGN 10
#define NTT2_COLS 128          // columns (threads) per CTA of an outer launch
#define NTT2_INNER_THREADS 64  // threads per CTA of an inner launch: one radix-16 group each
static inline bool ntt2_ok(int logn) { return logn >= 11 && logn <= 15; }

// R outer forward stages on one column held in registers (stage st pairs k and k + 2^(R-1-st);
// its twiddle index m + (k >> (R - st)) with m = 2^st does not depend on the column)
template <int R>
__device__ __forceinline__ void outer_fwd_regs(u64 (&v)[1 << R], const u64 *__restrict__ tw, u64 q) {
    const u64 q2 = 2 * q;
#pragma unroll
    for (int st = 0; st < R; ++st) {
        const int h = 1 << (R - 1 - st);
#pragma unroll
        for (int k0 = 0; k0 < (1 << R); k0 += 2 * h) {
            const ulonglong2 W = tw_fwd(tw, (1u << st) + (u32)(k0 >> (R - st)));
#pragma unroll
            for (int kk = 0; kk < h; ++kk) {
                u64 U = v[k0 + kk];
                if (U >= q2) U -= q2;
                const u64 V = shoup_lazy(v[k0 + kk + h], W.x, W.y, q);
                v[k0 + kk] = U + V;
                v[k0 + kk + h] = U - V + q2;
            }
        }
    }
}

// R outer inverse stages (distances 1024 * 2^b, b = 0 .. R-1) on one column, then the N^-1 factor
template <int R>
__device__ __forceinline__ void outer_inv_regs(u64 (&v)[1 << R], const u64 *__restrict__ tw, u32 N, u64 q,
                                               u64 ninv, u64 ninvs) {
    const u64 q2 = 2 * q;
#pragma unroll
    for (int b = 0; b < R; ++b) {
        const int d = 1 << b;
        const u32 hb = N >> (NTT2_INNER_LOGN + 1 + b);
#pragma unroll
        for (int k0 = 0; k0 < (1 << R); k0 += 2 * d) {
            const ulonglong2 W = tw_inv(tw, N, hb + (u32)(k0 >> (b + 1)));
#pragma unroll
            for (int kk = 0; kk < d; ++kk) {
                const u64 U = v[k0 + kk], V = v[k0 + kk + d];
                u64 sm = U + V;
                if (sm >= q2) sm -= q2;
                v[k0 + kk] = sm;
                v[k0 + kk + d] = shoup_lazy(U - V + q2, W.x, W.y, q);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) v[k] = mul_shoup(v[k], ninv, ninvs, q);
}

// the ten inner forward stages of the block at goff (held in sm by the caller), outputs in [0, q)
__device__ __forceinline__ void inner_fwd_block(u64 *sm, int logn, const u64 *__restrict__ tw, u64 q, u32 goff) {
    fwd_local(sm, logn, logn - NTT2_INNER_LOGN, tw, q, NTT2_INNER_LOGN, goff);
}
// the ten inner inverse stages of the block at goff (no N^-1 factor: the outer launch applies it)
__device__ __forceinline__ void inner_inv_block(u64 *sm, int logn, const u64 *__restrict__ tw, u64 q, u32 goff) {
    inv_local(sm, logn, NTT2_INNER_LOGN, tw, q, NTT2_INNER_LOGN, goff, false, 0, 0);
}

// launch the outer kernel template instance for R = logn - 10 (grid.x = rows, grid.y = column tiles)
#define NTT2_OUTER_LAUNCH(c, KERN, logn, rows, ...)                                                     \
    do {                                                                                                \
        const dim3 g__((rows), (1u << NTT2_INNER_LOGN) / NTT2_COLS);                                    \
        switch ((logn) - NTT2_INNER_LOGN) {                                                             \
            case 1: KERN<1><<<g__, NTT2_COLS, 0, (c)->stream>>>(__VA_ARGS__); break;                    \
            case 2: KERN<2><<<g__, NTT2_COLS, 0, (c)->stream>>>(__VA_ARGS__); break;                    \
            case 3: KERN<3><<<g__, NTT2_COLS, 0, (c)->stream>>>(__VA_ARGS__); break;                    \
            case 4: KERN<4><<<g__, NTT2_COLS, 0, (c)->stream>>>(__VA_ARGS__); break;                    \
            case 5: KERN<5><<<g__, NTT2_COLS, 0, (c)->stream>>>(__VA_ARGS__); break;                    \
            default: throw HeError(HE_EINVAL, "two-kernel NTT: ring degree out of range");             \
        }                                                                                               \
    } while (0)
