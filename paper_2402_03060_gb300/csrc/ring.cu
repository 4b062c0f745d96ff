// ring.cu -- elementwise ring kernels: modular add/sub/mul with batch
// broadcasting, Galois permutation, ciphertext tensor, counter-based samplers,
// and the plaintext-mask multiply-accumulate of the convolution / FC layers.
// All arrays are rows of N residues; the prime of row r is given by a regular
// map (w = r % period; prime = w < lp ? w : pbase + w - lp).
#include "ring.cuh"

__device__ __forceinline__ u32 map_prime(u32 r, u32 period, u32 lp, u32 pbase) {
    u32 w = r % period;
    return w < lp ? w : pbase + (w - lp);
}

// ---------------------------------------------------------------- binops
__global__ void binop_kernel(int op, u64 *out, const u64 *a, const u64 *b, u32 rows, u32 logn, u32 period, u32 lp,
                             u32 pbase, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * N) return;
    u32 r = (u32)(idx >> logn);
    const PrimeDev &P = pd[map_prime(r, period, lp, pbase)];
    u64 x = a[idx], y = b ? b[idx] : 0, z;
    switch (op) {
        case OP_ADD: z = add_mod(x, y, P.q); break;
        case OP_SUB: z = sub_mod(x, y, P.q); break;
        case OP_MUL: z = mul_mod(x, y, P); break;
        case OP_NEG: z = neg_mod(x, P.q); break;
        default: z = x;
    }
    out[idx] = z;
}

void ew_binop(Ctx *c, int op, u64 *out, const u64 *a, const u64 *b, u32 rows, u32 period, u32 lp, u32 pbase) {
    size_t total = (size_t)rows * c->N;
    if (!total) return;
    prof_begin(c);
    binop_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(op, out, a, b, rows, c->logn, period, lp,
                                                                        pbase, c->pdev);
    note_launch(c, "binop", 8.0 * total * (b ? 3 : 2));
}

// out[b][k][l][n] = a[b][k][l][n] (op) pt[l][n] for the polys k in kmask; other polys copied.
__global__ void bcast_kernel(int op, u64 *out, const u64 *a, const u64 *pt, u32 B, u32 lp, u32 logn, u32 kmask,
                             const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)B * 2 * lp * N;
    if (idx >= total) return;
    u32 n = (u32)(idx & (N - 1));
    size_t r = idx >> logn;
    u32 l = (u32)(r % lp);
    u32 k = (u32)((r / lp) & 1);
    u64 x = a[idx];
    if ((kmask >> k) & 1) {
        const PrimeDev &P = pd[l];
        u64 y = pt[(size_t)l * N + n];
        x = op == OP_MUL ? mul_mod(x, y, P) : add_mod(x, y, P.q);
    }
    out[idx] = x;
}

void ew_bcast(Ctx *c, int op, u64 *out, const u64 *a, const u64 *pt, u32 B, u32 lp, u32 kmask) {
    size_t total = (size_t)B * 2 * lp * c->N;
    if (!total) return;
    prof_begin(c);
    bcast_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(op, out, a, pt, B, lp, c->logn, kmask,
                                                                        c->pdev);
    note_launch(c, "bcast", 8.0 * (2.0 * total + (double)lp * c->N));
}

// out[o][b][0][l][n] += pt[o][l][n]   (bias of channel o, added to c0 of every ciphertext)
__global__ void add_plain_multi_kernel(u64 *out, const u64 *pt, u32 O, u32 B, u32 lp, u32 logn, size_t o_stride,
                                       const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)O * B * lp * N;
    if (idx >= total) return;
    u32 n = (u32)(idx & (N - 1));
    size_t r = idx >> logn;
    u32 l = (u32)(r % lp);
    size_t ob = r / lp;
    u32 b = (u32)(ob % B), o = (u32)(ob / B);
    u64 *p = out + o * o_stride + ((size_t)b * 2 * lp + l) * N + n;
    *p = add_mod(*p, pt[((size_t)o * lp + l) * N + n], pd[l].q);
}

void add_plain_multi(Ctx *c, u64 *out, const u64 *pt, u32 O, u32 B, u32 lp, size_t o_stride) {
    size_t total = (size_t)O * B * lp * c->N;
    if (!total) return;
    prof_begin(c);
    add_plain_multi_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, pt, O, B, lp, c->logn,
                                                                                  o_stride, c->pdev);
    note_launch(c, "add_plain");
}

// --------------------------------------------------------------- Galois
__global__ void perm_kernel(u64 *out, const u64 *in, u32 rows, u32 logn, u32 g) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * N) return;
    u32 n = (u32)(idx & (N - 1));
    size_t r = idx >> logn;
    out[idx] = in[r * N + galois_src(n, g, logn)];
}

void galois_permute(Ctx *c, u64 *out, const u64 *in, u32 rows, u32 g) {
    size_t total = (size_t)rows * c->N;
    if (!total) return;
    prof_begin(c);
    perm_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, in, rows, c->logn, g);
    note_launch(c, "galois");
}

// --------------------------------------------------------------- tensor
// d[b][0..2][l] = (a0*a0, 2*a0*a1, a1*a1)
__global__ void tensor_sq_kernel(u64 *d, const u64 *a, u32 B, u32 lp, u32 logn, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)B * lp * N;
    if (idx >= total) return;
    u32 n = (u32)(idx & (N - 1));
    size_t r = idx >> logn;
    u32 l = (u32)(r % lp);
    u32 b = (u32)(r / lp);
    const PrimeDev &P = pd[l];
    const u64 *ab = a + (size_t)b * 2 * lp * N;
    u64 a0 = ab[(size_t)l * N + n], a1 = ab[(size_t)(lp + l) * N + n];
    u64 m01 = mul_mod(a0, a1, P);
    u64 *db = d + (size_t)b * 3 * lp * N;
    db[(size_t)l * N + n] = mul_mod(a0, a0, P);
    db[(size_t)(lp + l) * N + n] = add_mod(m01, m01, P.q);
    db[(size_t)(2 * lp + l) * N + n] = mul_mod(a1, a1, P);
}

void tensor_square(Ctx *c, u64 *d, const u64 *a, u32 B, u32 lp) {
    size_t total = (size_t)B * lp * c->N;
    prof_begin(c);
    tensor_sq_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(d, a, B, lp, c->logn, c->pdev);
    note_launch(c, "tensor");
}

// --------------------------------------------------------------- samplers
// Small polynomial (ternary or centred binomial eta=21): vector v draws word n
// of stream (seeds.seed[v], seeds.stream[v]); the value is reduced into every
// row's prime: out[v][row][n].
__global__ void sample_small_kernel(u64 *out, SeedList sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase,
                                   int kind, u32 logn, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nvec * N) return;
    u32 n = (u32)(idx & (N - 1));
    u32 v = (u32)(idx >> logn);
    u64 w = sm64_word(sm64_state(sl.seed[v], sl.stream[v]), n);
    i64 x;
    if (kind == 0) {
        x = (i64)(w % 3) - 1;
    } else {
        x = (i64)__popcll(w & 0x1FFFFFULL) - (i64)__popcll((w >> 21) & 0x1FFFFFULL);
    }
    for (u32 r = 0; r < rows; ++r) {
        const PrimeDev &P = pd[map_prime(r, period, lp, pbase)];
        u64 y = x >= 0 ? (u64)x : P.q - (u64)(-x);
        out[((size_t)v * rows + r) * N + n] = y;
    }
}

void sample_small(Ctx *c, u64 *out, const SeedList &sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase,
                  int kind) {
    if (nvec > SEEDLIST_MAX) throw HeError(HE_EINVAL, "sample_small: too many vectors");
    size_t total = (size_t)nvec * c->N;
    prof_begin(c);
    sample_small_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, sl, nvec, rows, period, lp,
                                                                               pbase, kind, c->logn, c->pdev);
    note_launch(c, "sample_small");
}

// Uniform residues: row r of vector v uses stream (seed[v], stream[v] + prime(r));
// value = floor(w * q / 2^64).
__global__ void sample_uniform_kernel(u64 *out, SeedList sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase,
                                     u32 logn, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nvec * rows * N) return;
    u32 n = (u32)(idx & (N - 1));
    u32 R = (u32)(idx >> logn);
    u32 r = R % rows, v = R / rows;
    u32 pr = map_prime(r, period, lp, pbase);
    const PrimeDev &P = pd[pr];
    out[idx] = mulhi64(sm64_word(sm64_state(sl.seed[v], sl.stream[v] + pr), n), P.q);
}

void sample_uniform(Ctx *c, u64 *out, const SeedList &sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase) {
    if (nvec > SEEDLIST_MAX) throw HeError(HE_EINVAL, "sample_uniform: too many vectors");
    size_t total = (size_t)nvec * rows * c->N;
    prof_begin(c);
    sample_uniform_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, sl, nvec, rows, period, lp,
                                                                                 pbase, c->logn, c->pdev);
    note_launch(c, "sample_uniform");
}

// --------------------------------------------------------------- MAC
// out[o][b][k][l][n] = sum_t pt[o][t][l][n] * x[t][b][k][l][n]   (mod q_l)
//
// A CTA owns NT consecutive coefficients of one limb and 256/NT
// (ciphertext, poly) pairs; it stages the plaintext tile pt[0..O)[t-chunk][l][n-tile]
// in shared memory once and every thread reuses it for its own pair, so a
// plaintext word is read from global memory once per 256/NT pairs instead of
// once per pair.  The tiles are double-buffered: the copies of tile k+1 are issued
// when tile k starts and land while it is computed.  Lanes of a warp cover 4+
// consecutive coefficients of 8 or fewer pairs, so every ciphertext load is a full
// 32-byte sector.  Each thread keeps all O sums as 128-bit accumulators (products
// < 2^120, folded every 128 terms).
#define MAC_DEPTH 8
// OSPLIT threads share one (ciphertext, poly, coefficient): each keeps OMAX of the launch's
// OMAX * OSPLIT outputs (fewer registers, more resident warps; the second thread's
// ciphertext loads hit L1)
template <int OMAX, int OSPLIT>
__global__ void __launch_bounds__(256, OSPLIT == 1 ? 2 : 3) mac_kernel(u64 *out, const u64 *__restrict__ x, const u64 *__restrict__ pt,
                                                  u32 O, u32 T, u32 BK, u32 lp, u32 logn, size_t x_tstride,
                                                  size_t out_ostride, u32 ntlog, u32 tc, u32 lpq, u32 pbase,
                                                  int accumulate, size_t pt_ostride, u32 l0,
                                                  const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 smem[];
    u64 *xs = smem;                          // [256][MAC_DEPTH]: each thread's own pipeline slots
    u64 *ps0 = smem + 256 * MAC_DEPTH;       // two plaintext tiles, each [tc][NT][OW]
    constexpr u32 OW = OMAX * OSPLIT;
    const u32 N = 1u << logn, NT = 1u << ntlog;
    const u32 tid = threadIdx.x;
    const u32 osub = tid % OSPLIT, rt = tid / OSPLIT;
    const u32 nl = rt & (NT - 1);
    const u32 bk = blockIdx.x * ((256u / OSPLIT) >> ntlog) + (rt >> ntlog);
    const u32 n0 = blockIdx.y * NT;
    const u32 l = l0 + blockIdx.z;
    const bool active = bk < BK;
    const PrimeDev P = pd[l < lpq ? l : pbase + (l - lpq)];
    Acc128 acc[OMAX];
#pragma unroll
    for (int o = 0; o < OMAX; ++o) acc[o].lo = acc[o].hi = 0;
    const size_t xoff = ((size_t)bk * lp + l) * N + n0 + nl;   // bk = b*2 + k
    const size_t pstride_t = (size_t)lp * N;
    const size_t tile_words = (size_t)tc * NT * OW;
    u64 *myx = xs + tid * MAC_DEPTH;
    // the plaintext words of terms [t0, t0 + tc) into dst, every word in flight at once
    // (one commit group)
    auto load_tile = [&](u32 t0, u64 *dst) {
        const u32 tcc = T - t0 < tc ? T - t0 : tc;
        for (u32 idx = tid; idx < O * tcc * NT; idx += blockDim.x) {
            const u32 j = idx & (NT - 1), r = idx >> ntlog;
            const u32 tt = r % tcc, o = r / tcc;
            cp_async8(dst + (tt * NT + j) * OW + o,
                      pt + (size_t)o * pt_ostride + (size_t)(t0 + tt) * pstride_t + (size_t)l * N + n0 + j);
        }
        cp_commit();
    };
    // prologue: the first MAC_DEPTH terms in flight (one commit group per term), then tile 0
#pragma unroll
    for (int d = 0; d < MAC_DEPTH; ++d) {
        if (active && (u32)d < T) cp_async8(myx + d, x + (size_t)d * x_tstride + xoff);
        cp_commit();
    }
    load_tile(0, ps0);
    u32 cnt = 0, k = 0;
    for (u32 t0 = 0; t0 < T; t0 += tc, ++k) {
        const u32 tcc = T - t0 < tc ? T - t0 : tc;
        const u64 *ps = ps0 + (k & 1) * tile_words;
        // this thread's copies of tile k are older than the newest MAC_DEPTH - 1 commit
        // groups once the previous (full) tile ran at least that many terms (one group per term)
        if (k > 0 && tc >= MAC_DEPTH - 1)
            cp_wait<MAC_DEPTH - 1>();
        else
            cp_wait<0>();
        // every thread's copies of tile k are visible and every thread is done with tile
        // k-1, whose buffer now receives tile k+1
        __syncthreads();
        if (t0 + tc < T) load_tile(t0 + tc, ps0 + ((k + 1) & 1) * tile_words);
        for (u32 tt = 0; tt < tcc; ++tt) {
            const u32 t = t0 + tt;
            cp_wait<MAC_DEPTH - 1>();        // the copy of term t has landed
            const u64 xv = myx[t % MAC_DEPTH];
            if (active) {
                // this thread's OMAX plaintext words of term t, 16-byte loads at fixed offsets
                const u64 *pw0 = ps + (tt * NT + nl) * OW + osub * OMAX;
                const ulonglong2 *pv = reinterpret_cast<const ulonglong2 *>(pw0);
                u64 pw[OMAX];
#pragma unroll
                for (int o = 0; o < OMAX / 2; ++o) {
                    const ulonglong2 v = pv[o];
                    pw[2 * o] = v.x;
                    pw[2 * o + 1] = v.y;
                }
                if (OMAX & 1) pw[OMAX - 1] = pw0[OMAX - 1];
#pragma unroll
                for (int o = 0; o < OMAX; ++o) mac128(acc[o], pw[o], xv);
            }
            if (active && t + MAC_DEPTH < T) cp_async8(myx + t % MAC_DEPTH, x + (size_t)(t + MAC_DEPTH) * x_tstride + xoff);
            cp_commit();
            if (++cnt == 128) {
                cnt = 0;
#pragma unroll
                for (int o = 0; o < OMAX; ++o) {
                    acc[o].lo = reduce128(acc[o].lo, acc[o].hi, P);
                    acc[o].hi = 0;
                }
            }
        }
    }
    cp_wait<0>();
    if (!active) return;
#pragma unroll
    for (int o = 0; o < OMAX; ++o)
        if (osub * OMAX + o < O) {
            u64 *dst = out + (osub * OMAX + o) * out_ostride + xoff;
            if (accumulate) mac128(acc[o], *dst, 1);
            *dst = reduce128(acc[o].lo, acc[o].hi, P);
        }
}

// The same sums for one or two outputs: one thread per (ciphertext, poly, limb, coefficient),
// no shared-memory tile (nothing to share between polynomials when O <= 2), loads unrolled
// four terms deep; a memory-bound kernel that keeps the whole GPU occupied.
template <int OM>
__global__ void __launch_bounds__(256) mac_small_kernel(u64 *out, const u64 *__restrict__ x,
                                                        const u64 *__restrict__ pt, u32 O, u32 T, u32 BK, u32 lp,
                                                        u32 logn, size_t x_tstride, size_t out_ostride, u32 lpq,
                                                        u32 pbase, int accumulate, size_t pt_ostride,
                                                        const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)BK * lp * N) return;
    const u32 n = (u32)(idx & (N - 1));
    const size_t r = idx >> logn;
    const u32 l = (u32)(r % lp), bk = (u32)(r / lp);
    const PrimeDev P = pd[l < lpq ? l : pbase + (l - lpq)];
    const size_t xoff = ((size_t)bk * lp + l) * N + n;
    const size_t poff = (size_t)l * N + n, pstride_t = (size_t)lp * N;
    Acc128 acc[OM];
#pragma unroll
    for (int o = 0; o < OM; ++o) acc[o].lo = acc[o].hi = 0;
    u32 t = 0;
    while (t < T) {
        const u32 tend = T - t > 128 ? t + 128 : T;   // fold every 128 terms (products < 2^120)
#pragma unroll 4
        for (; t < tend; ++t) {
            const u64 xv = __ldg(x + (size_t)t * x_tstride + xoff);
#pragma unroll
            for (int o = 0; o < OM; ++o)
                if (o < (int)O) mac128(acc[o], __ldg(pt + (size_t)o * pt_ostride + (size_t)t * pstride_t + poff), xv);
        }
        if (t < T) {
#pragma unroll
            for (int o = 0; o < OM; ++o) {
                acc[o].lo = reduce128(acc[o].lo, acc[o].hi, P);
                acc[o].hi = 0;
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OM; ++o)
        if (o < (int)O) {
            u64 *dst = out + o * out_ostride + xoff;
            if (accumulate) mac128(acc[o], *dst, 1);
            *dst = reduce128(acc[o].lo, acc[o].hi, P);
        }
}

void mac_init(Ctx *c) {
    (void)c;
    for (const void *f : {(const void *)mac_kernel<1, 1>, (const void *)mac_kernel<2, 1>,
                          (const void *)mac_kernel<4, 1>, (const void *)mac_kernel<6, 1>,
                          (const void *)mac_kernel<8, 1>, (const void *)mac_kernel<12, 1>,
                          (const void *)mac_kernel<6, 2>})
        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
}

#define MAC_TC_TMAX 112   // terms of one tensor-core MAC launch (the exactness bound below)
static void mac_tc(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O, u32 T,
                   u32 B, u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride, u32 l0, u32 nl);
static u32 mac_tc_bytes(const Ctx *c, u32 p);
static void mac_int(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O,
                    u32 T, u32 B, u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride, u32 l0, u32 nl);

void mac(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O, u32 T, u32 B,
         u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride) {
    if (!pt_ostride) pt_ostride = (size_t)T * lp * c->N;
    // pt [O][T][lp][N]; x [T] blocks of [B][2][lp][N] at x_tstride; out [O] blocks at out_ostride.
    // Limb l < lpq uses data prime l, limb l >= lpq special prime pbase + l - lpq.
    if (lpq == ~0u) lpq = lp;
    const int tcmax = tune_get(c, TUNE_MAC_TC, 0);   // limbs of at most this many bytes on the tensor cores
    // the tensor form takes 6 to 16 outputs and at most MAC_TC_TMAX terms (one product launch)
    if (O < 6 || O > 16 || T > MAC_TC_TMAX || tcmax <= 0) {
        mac_int(c, out, out_ostride, x, x_tstride, pt, O, T, B, lp, lpq, pbase, accumulate, pt_ostride, 0, lp);
        return;
    }
    // runs of consecutive limbs on the same units
    for (u32 l0 = 0; l0 < lp;) {
        auto on_tc = [&](u32 l) { return (int)mac_tc_bytes(c, l < lpq ? l : pbase + (l - lpq)) <= tcmax; };
        const bool tc = on_tc(l0);
        u32 l1 = l0 + 1;
        while (l1 < lp && on_tc(l1) == tc) ++l1;
        if (tc)
            mac_tc(c, out, out_ostride, x, x_tstride, pt, O, T, B, lp, lpq, pbase, accumulate, pt_ostride, l0, l1 - l0);
        else
            mac_int(c, out, out_ostride, x, x_tstride, pt, O, T, B, lp, lpq, pbase, accumulate, pt_ostride, l0, l1 - l0);
        l0 = l1;
    }
}

// mac() on the integer units over the limbs [l0, l0 + nl)
static void mac_int(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O,
                    u32 T, u32 B, u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride, u32 l0, u32 nl) {
    const u32 BK = 2 * B;
    if (O <= 2) {
        const size_t total = (size_t)BK * lp * c->N;
        prof_begin(c);
        if (O == 1)
            mac_small_kernel<1><<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(
                out, x, pt, O, T, BK, lp, c->logn, x_tstride, out_ostride, lpq, pbase, accumulate, pt_ostride, c->pdev);
        else
            mac_small_kernel<2><<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(
                out, x, pt, O, T, BK, lp, c->logn, x_tstride, out_ostride, lpq, pbase, accumulate, pt_ostride, c->pdev);
        note_launch(c, "mac", 8.0 * c->N * ((double)O * T * lp + (double)T * B * 2 * lp + (double)O * B * 2 * lp),
                    (double)O * T * B * 2 * lp * c->N);
        return;
    }
    const u32 bk_max = (u32)tune_get(c, TUNE_MAC_BK, 64);   // polynomials per CTA (tuned: 16, 32, 64)
    // outputs in groups of at most G (the accumulators of a group live in registers;
    // every group re-reads the inputs x); G is tuned, 12 by default.  With the split
    // knob a group of more than 6 outputs is shared by two threads per coefficient.
    const u32 G = (u32)tune_get(c, TUNE_MAC_GROUP, 12);
    const u32 split = (u32)tune_get(c, TUNE_MAC_SPLIT, 1);
    for (u32 o0 = 0; o0 < O; o0 += G) {
        const u32 oc = O - o0 < G ? O - o0 : G;
        const u32 os = split == 2 && oc > 6 && oc <= 12 ? 2 : 1;
        u32 bkc = 1;
        while (bkc < BK && bkc < bk_max / os) bkc <<= 1;
        u32 ntlog = 0;
        while ((1u << ntlog) * bkc * os < 256) ++ntlog;
        if ((1u << ntlog) > c->N) throw HeError(HE_EINVAL, "mac: ring too small");
        const u32 NT = 1u << ntlog;
        // shared memory: pipeline slots (16 KB) + two plaintext tiles of at most 40 KB each
        // (28 KB with the split, which keeps three CTAs per SM)
        const u32 ow = os == 2 ? 12 : oc <= 1 ? 1 : oc <= 2 ? 2 : oc <= 4 ? 4 : oc <= 6 ? 6 : oc <= 8 ? 8 : 12;
        u32 tc = (os == 2 ? 3584u : 5120u) / (ow * NT);
        if (tc < 1) tc = 1;
        if (tc > T) tc = T;
        const size_t smem = (2 * (size_t)ow * tc * NT + 256 * MAC_DEPTH) * 8;
        dim3 grid((BK + bkc - 1) / bkc, c->N / NT, nl);
        const u64 *ptc = pt + (size_t)o0 * pt_ostride;
        u64 *outc = out + (size_t)o0 * out_ostride;
        prof_begin(c);
#define MAC_LAUNCH(OM, OS)                                                                                        \
    mac_kernel<OM, OS><<<grid, 256, smem, c->stream>>>(outc, x, ptc, oc, T, BK, lp, c->logn, x_tstride, out_ostride, \
                                                       ntlog, tc, lpq, pbase, accumulate, pt_ostride, l0, c->pdev)
        if (os == 2)
            MAC_LAUNCH(6, 2);
        else if (oc <= 1)
            MAC_LAUNCH(1, 1);
        else if (oc <= 2)
            MAC_LAUNCH(2, 1);
        else if (oc <= 4)
            MAC_LAUNCH(4, 1);
        else if (oc <= 6)
            MAC_LAUNCH(6, 1);
        else if (oc <= 8)
            MAC_LAUNCH(8, 1);
        else
            MAC_LAUNCH(12, 1);
#undef MAC_LAUNCH
        note_launch(c, "mac", 8.0 * c->N * ((double)oc * T * nl + (double)T * B * 2 * nl + (double)oc * B * 2 * nl),
                    (double)oc * T * B * 2 * nl * c->N);
    }
}

// --------------------------------------------------------------- tensor-core MAC
// The same sums out[o][c] (+)= sum_{t<T} pt[o][t] (.) x[t][c] (mod q_l, c = 2b + k a column), per
// coefficient n and limb l a matrix product W (O x T) X (T x columns), on the tensor cores
// (mma.sync m16n8k16, fp16 operands, fp32 accumulation).  A residue v < 256^C (C = the bytes of
// q_l) is written v = sum_{a<C} d_a 256^a + Cc with d_a = (byte a of v) - 128 in [-128, 127],
// exact in fp16, and Cc = 128 (256^C - 1) / 255.  Then
//   sum_t w_t x_t = sum_{k<2C-1} 2^(8k) S_k + Cc sum_t w_t + Cc sum_t x_t - T' Cc^2,
//   S_k = sum_{a+b=k} sum_t e_a(w_t) d_b(x_t)      (e, d the digits of w, x)
// over the T' = 16 * ceil(T / 16) terms staged (the padding terms are zeros on both sides and
// drop out of the identity).  |e d| <= 2^14 and a shift collects at most C <= 8 digit pairs, so
// with T' <= MAC_TC_TMAX every partial sum of S_k is an integer below 2^24 in magnitude: the fp32
// accumulation is exact.  The S_k are assembled in 128-bit integers and reduced mod q.
//
// The masks are decomposed first (mac_tc_prep_kernel): their digits in the A-fragment order of
// every lane, and sum_t w_t, per coefficient.  CTA of the product: one limb, 4 consecutive
// coefficients, 32 columns; 16 warps, warp w takes coefficient w / 4 and the 8-column tile w % 4
// (an m16n8 tile: outputs on the rows) and loads its mask fragments straight from the digit
// buffer (16 bytes per lane).  The x terms stream in chunks of 16 through three shared-memory
// stages filled by cp.async (4 consecutive lanes copy the 4 coefficients of one row: full
// 32-byte sectors), one barrier per chunk; rows are 16 terms + 8 words of padding, so the
// 16-byte fragment reads of a warp are free of bank conflicts.  The column sums sum_t x_t are
// taken by the lanes from the words of their own fragments.
#define MAC_TC_ROW 24                                         // words per staged row (16 terms + pad)
#define MAC_TC_XS (4 * 32 * MAC_TC_ROW)                       // x stage: [4 n][32 columns][row]
#define MAC_TC_STAGES 3
#define MAC_TC_SMEM ((size_t)MAC_TC_STAGES * MAC_TC_XS * 8)
#define MAC_TC_TAB 20                                         // constants per prime

__device__ __forceinline__ void cp_async8_zfill(u64 *smem, const u64 *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;   // 0: nothing read, the destination is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

// digit a of v0 and of v1 as an fp16 pair (low half v0): (byte | 0x6400) is 1024 + byte in fp16
__device__ __forceinline__ u32 tc_digits(u64 v0, u64 v1, int a) {
    const u32 w0 = a < 4 ? (u32)v0 : (u32)(v0 >> 32), w1 = a < 4 ? (u32)v1 : (u32)(v1 >> 32);
    const u32 p = (__byte_perm(w0, w1, (u32)(a & 3) | ((u32)(4 + (a & 3)) << 8)) & 0x00ff00ffu) | 0x64006400u;
    u32 r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(p), "r"(0x64806480u));   // - 1152 = - (1024 + 128)
    return r;
}

__device__ __forceinline__ void mma_16816(float *d, const u32 *a, u32 b0, u32 b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (lo, hi) += s * c, s < 2^32, c < 2^64
__device__ __forceinline__ void mac_u32(u64 &lo, u64 &hi, u32 s, u64 c) {
    const u64 pl = (u64)s * (u32)c, ph = (u64)s * (u32)(c >> 32);
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, 0;\n\t"
        "add.cc.u64 %0, %0, %3;\n\t"
        "addc.u64 %1, %1, %4;"
        : "+l"(lo), "+l"(hi)
        : "l"(pl), "l"(ph << 32), "l"(ph >> 32));
}

// The mask digits of one launch: wd [nl][N/4][nk][4][CS][32 lanes][4] u32 (CS digit slots, C of
// the limb used) holding, for chunk kc, coefficient n0 + nn and digit a, the A fragment of lane
// (g, tg): (w[g][t], w[g][t+1]), (w[g+8][t], ..), (w[g][t+8], ..), (w[g+8][t+8], ..), t = 16 kc +
// 2 tg, zeros beyond O outputs and T terms; wsum [nl][16][N] = sum_t w[o][t] mod q.  Grid
// (N / 4, nl), 512 threads: thread (nn, lane, reg) = (tid / 128, tid / 4 % 32, tid % 4).
__global__ void __launch_bounds__(512) mac_tc_prep_kernel(u32 *wd, u64 *wsum, const u64 *__restrict__ pt, u32 O,
                                                          u32 T, u32 lp, u32 l0, u32 logn, size_t pt_ostride,
                                                          u32 CS, u32 lpq, u32 pbase, const u64 *__restrict__ tctab,
                                                          const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 nb = blockIdx.x, lr = blockIdx.y, l = l0 + lr, n0 = nb * 4;
    const u32 p = l < lpq ? l : pbase + (l - lpq);
    const int C = (int)tctab[(size_t)p * MAC_TC_TAB];
    const u64 q = pd[p].q;
    const u32 tid = threadIdx.x, nn = tid >> 7, lane = (tid >> 2) & 31, r = tid & 3;
    const u32 o = (lane >> 2) + (r & 1) * 8, tr = 2 * (lane & 3) + (r >> 1) * 8;
    const u32 nk = (T + 15) / 16;
    const size_t lstride = (size_t)lp * N;
    const u64 *w = o < O ? pt + (size_t)o * pt_ostride + (size_t)l * N + n0 + nn : pt;
    u32 *dst = wd + ((size_t)lr * (N / 4) + nb) * nk * 4 * CS * 128 + (nn * CS * 32 + lane) * 4 + r;
    for (u32 kc = 0; kc < nk; ++kc) {
        const u32 t = kc * 16 + tr;
        const u64 v0 = o < O && t < T ? w[(size_t)t * lstride] : 0;
        const u64 v1 = o < O && t + 1 < T ? w[(size_t)(t + 1) * lstride] : 0;
        for (int a = 0; a < C; ++a) dst[((size_t)kc * 4 * CS + a) * 128] = tc_digits(v0, v1, a);
    }
    if (tid < 64) {   // (o, nn) = (tid % 16, tid / 16)
        const u32 os = tid & 15, ns = tid >> 4;
        u64 sum = 0;
        if (os < O) {
            const u64 *ws = pt + (size_t)os * pt_ostride + (size_t)l * N + n0 + ns;
            for (u32 t = 0; t < T; ++t) sum = add_mod(sum, ws[(size_t)t * lstride], q);
        }
        wsum[((size_t)lr * 16 + os) * N + n0 + ns] = sum;
    }
}

template <int C>
__device__ __forceinline__ void mac_tc_body(u64 *out, const u64 *__restrict__ x, const u32 *__restrict__ wd,
                                            const u64 *__restrict__ wsum, u32 O, u32 T, u32 BK, u32 lp, u32 l,
                                            u32 lr, u32 logn, size_t x_tstride, size_t out_ostride, u32 CS,
                                            int accumulate, const PrimeDev &P, const u64 *__restrict__ tab,
                                            u64 *smem) {
    constexpr int NS = 2 * C - 1;
    const u32 N = 1u << logn;
    const u32 nb = blockIdx.y, n0 = nb * 4, col0 = blockIdx.x * 32;
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 g = lane >> 2, tg = lane & 3, nn = warp >> 2, ct = warp & 3;
    const u32 nk = (T + 15) / 16;
    const size_t lstride = (size_t)lp * N;   // one column to the next

    // this thread's copies, the same offsets every chunk: x rows (n, col) of terms tid/128 + 4r
    const u32 xn = tid & 3, xcol = (tid >> 2) & 31, xt = tid >> 7;
    const bool xok = col0 + xcol < BK;
    const u64 *xsrc = x + (size_t)xt * x_tstride + (size_t)(col0 + xcol) * lstride + (size_t)l * N + n0 + xn;
    const size_t xstep = 4 * x_tstride;
    auto issue = [&](u32 kc) {
        u64 *xs = smem + (kc % MAC_TC_STAGES) * MAC_TC_XS;
        const u32 t0 = kc * 16;
        const u64 *xp = xsrc + (size_t)t0 * x_tstride;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool ok = xok && t0 + xt + 4 * r < T;
            cp_async8_zfill(xs + (xn * 32 + xcol) * MAC_TC_ROW + xt + 4 * r, ok ? xp + r * xstep : x, ok);
        }
    };
    const u32 *wdl = wd + ((size_t)lr * (N / 4) + nb) * nk * 4 * CS * 128 + (nn * CS * 32 + lane) * 4;

    float acc[NS][4];
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
    u64 slo = 0, shi = 0;   // 128-bit sum of this lane's x words: column 8ct + g, four terms a chunk
    issue(0);
    cp_commit();
    if (nk > 1) issue(1);
    cp_commit();
    for (u32 kc = 0; kc < nk; ++kc) {
        cp_wait<1>();
        __syncthreads();   // chunk kc staged for every thread; chunk kc-1's stage is free
        if (kc + 2 < nk) issue(kc + 2);
        cp_commit();
        const u64 *xs = smem + (kc % MAC_TC_STAGES) * MAC_TC_XS;
        // B fragments: the digits of x[t][col] for t = 2tg, 2tg+1 (b0) and 2tg+8, 2tg+9 (b1), col = 8ct + g
        const u64 *xr = xs + (nn * 32 + ct * 8 + g) * MAC_TC_ROW;
        const ulonglong2 xa = *reinterpret_cast<const ulonglong2 *>(xr + 2 * tg);
        const ulonglong2 xb = *reinterpret_cast<const ulonglong2 *>(xr + 2 * tg + 8);
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;\n\t"
            "add.cc.u64 %0, %0, %3;\n\taddc.u64 %1, %1, 0;\n\t"
            "add.cc.u64 %0, %0, %4;\n\taddc.u64 %1, %1, 0;\n\t"
            "add.cc.u64 %0, %0, %5;\n\taddc.u64 %1, %1, 0;"
            : "+l"(slo), "+l"(shi)
            : "l"(xa.x), "l"(xa.y), "l"(xb.x), "l"(xb.y));
        u32 bf[C][2];
#pragma unroll
        for (int b = 0; b < C; ++b) {
            bf[b][0] = tc_digits(xa.x, xa.y, b);
            bf[b][1] = tc_digits(xb.x, xb.y, b);
        }
        const u32 *wk = wdl + (size_t)kc * 4 * CS * 128;
#pragma unroll
        for (int a = 0; a < C; ++a) {
            const uint4 av = __ldg(reinterpret_cast<const uint4 *>(wk + a * 128));
            const u32 af[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
            for (int b = 0; b < C; ++b) mma_16816(acc[a + b], af, bf[b][0], bf[b][1]);
        }
    }
    // column sums: the four lanes of a column (same g) hold its terms; then lane (g, tg) takes
    // the sums of its output columns 2tg and 2tg + 1 from the lanes that hold them
    u64 xsum = reduce128(slo, shi, P);
    xsum = add_mod(xsum, __shfl_xor_sync(0xffffffffu, xsum, 1), P.q);
    xsum = add_mod(xsum, __shfl_xor_sync(0xffffffffu, xsum, 2), P.q);
    const u64 xs0 = __shfl_sync(0xffffffffu, xsum, (2 * tg) * 4), xs1 = __shfl_sync(0xffffffffu, xsum, (2 * tg + 1) * 4);
    // u_k = S_k + 2^24 >= 0, three shifts at a time combined in 64 bits (< 2^42) and multiplied by
    // 2^(8k) mod q into a 128-bit sum (< 5 * 2^103), reduced; then - 2^24 sum_k 2^(8k)
    // + Cc (sum w + sum x) - T' Cc^2
    const u64 q = P.q;
    const u64 tcc2 = mul_mod((u64)(nk * 16) % q, tab[MAC_TC_TAB - 1], P);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const u32 o = g + (e >> 1) * 8, col = col0 + ct * 8 + 2 * tg + (e & 1);
        if (o >= O || col >= BK) continue;
        Acc128 sum = {0, 0};
#pragma unroll
        for (int k0 = 0; k0 < NS; k0 += 3) {
            u64 v = 0;
#pragma unroll
            for (int j = 2; j >= 0; --j)
                if (k0 + j < NS) v = (v << 8) + (u64)(u32)(__float2int_rn(acc[k0 + j][e]) + (1 << 24));
            mac128(sum, v, tab[1 + k0]);
        }
        u64 r = sub_mod(reduce128(sum.lo, sum.hi, P), tab[16], q);
        const u64 sw = add_mod(wsum[((size_t)lr * 16 + o) * N + n0 + nn], (e & 1) ? xs1 : xs0, q);
        r = add_mod(r, mul_shoup(sw, tab[17], tab[18], q), q);
        r = sub_mod(r, tcc2, q);
        u64 *dst = out + (size_t)o * out_ostride + (size_t)col * lstride + (size_t)l * N + n0 + nn;
        if (accumulate) r = add_mod(r, *dst, q);
        *dst = r;
    }
}

__global__ void __launch_bounds__(512, 1) mac_tc_kernel(u64 *out, const u64 *__restrict__ x, const u32 *__restrict__ wd,
                                                        const u64 *__restrict__ wsum, u32 O, u32 T, u32 BK, u32 lp,
                                                        u32 l0, u32 logn, size_t x_tstride, size_t out_ostride,
                                                        u32 CS, u32 lpq, u32 pbase, int accumulate,
                                                        const u64 *__restrict__ tctab,
                                                        const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 smem[];
    const u32 lr = blockIdx.z, l = l0 + lr;
    const u32 p = l < lpq ? l : pbase + (l - lpq);
    const PrimeDev P = pd[p];
    const u64 *tab = tctab + (size_t)p * MAC_TC_TAB;
    switch ((int)tab[0]) {
#define MAC_TC_CASE(CV)                                                                                         \
    case CV:                                                                                                    \
        mac_tc_body<CV>(out, x, wd, wsum, O, T, BK, lp, l, lr, logn, x_tstride, out_ostride, CS, accumulate, P, \
                        tab, smem);                                                                             \
        break;
        MAC_TC_CASE(1) MAC_TC_CASE(2) MAC_TC_CASE(3) MAC_TC_CASE(4)
        MAC_TC_CASE(5) MAC_TC_CASE(6) MAC_TC_CASE(7) MAC_TC_CASE(8)
#undef MAC_TC_CASE
        default: break;
    }
}

// per prime: C (bytes of q), 2^(8k) mod q (k < 15), 2^24 sum_{k<2C-1} 2^(8k) mod q, Cc mod q with
// its Shoup companion, Cc^2 mod q
static const u64 *mac_tc_table(Ctx *c) {
    auto it = c->cache.find("mac_tc");
    if (it != c->cache.end()) return it->second.p;
    const size_t np = c->primes.size();
    std::vector<u64> h(np * MAC_TC_TAB, 0);
    for (size_t p = 0; p < np; ++p) {
        const u64 q = c->primes[p];
        const int bits = 64 - __builtin_clzll(q), C = (bits + 7) / 8;
        u64 *t = h.data() + p * MAC_TC_TAB;
        t[0] = (u64)C;
        unsigned __int128 pw = 1 % q, zs = 0;
        for (int k = 0; k < 15; ++k) {
            t[1 + k] = (u64)pw;
            if (k < 2 * C - 1) zs = (zs + pw) % q;
            pw = (pw << 8) % q;
        }
        t[16] = (u64)(((zs << 24)) % q);
        unsigned __int128 cc = 0;   // 128 * sum_{a<C} 256^a
        for (int a = 0; a < C; ++a) cc = (cc << 8) + 128;
        const u64 ccq = (u64)(cc % q);
        t[17] = ccq;
        t[18] = (u64)(((unsigned __int128)ccq << 64) / q);
        t[19] = (u64)((unsigned __int128)ccq * ccq % q);
    }
    return c->const_table("mac_tc", h);
}

void mac_tc_init() {
    CUDA_TRY(cudaFuncSetAttribute((const void *)mac_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)MAC_TC_SMEM));
}

static u32 mac_tc_bytes(const Ctx *c, u32 p) {
    const int bits = 64 - __builtin_clzll(c->primes[p]);
    return (u32)(bits + 7) / 8;
}

// mac() on the tensor cores over the limbs [l0, l0 + nl), O <= 16 outputs and T <= MAC_TC_TMAX
// terms: the decomposition of the masks, then the product
static void mac_tc(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O, u32 T,
                   u32 B, u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride, u32 l0, u32 nl) {
    const u32 BK = 2 * B, N = c->N, nk = (T + 15) / 16;
    if (N < 4) throw HeError(HE_EINVAL, "mac: ring too small");
    if (O > 16 || T > MAC_TC_TMAX) throw HeError(HE_EINVAL, "mac: more outputs or terms than one tensor-core launch");
    const u64 *tab = mac_tc_table(c);
    u32 CS = 1;   // digit slots: the largest prime of the limbs
    for (u32 l = l0; l < l0 + nl; ++l) CS = std::max(CS, mac_tc_bytes(c, l < lpq ? l : pbase + (l - lpq)));
    const size_t wd_u32 = (size_t)nl * N * nk * CS * 128;   // [nl][N/4][nk][4][CS][32][4]
    DBuf wd(c, (wd_u32 + 1) / 2);
    DBuf ws(c, (size_t)nl * 16 * N);
    prof_begin(c);
    mac_tc_prep_kernel<<<dim3(N / 4, nl), 512, 0, c->stream>>>(reinterpret_cast<u32 *>(wd.p), ws.p, pt, O, T, lp, l0,
                                                              c->logn, pt_ostride, CS, lpq, pbase, tab, c->pdev);
    note_launch(c, "mac_prep", 8.0 * N * ((double)O * T * nl + 16.0 * nl) + 4.0 * (double)wd_u32);
    const dim3 grid((BK + 31) / 32, N / 4, nl);
    prof_begin(c);
    mac_tc_kernel<<<grid, 512, MAC_TC_SMEM, c->stream>>>(out, x, reinterpret_cast<const u32 *>(wd.p), ws.p, O, T, BK,
                                                         lp, l0, c->logn, x_tstride, out_ostride, CS, lpq, pbase,
                                                         accumulate, tab, c->pdev);
    note_launch(c, "mac", 8.0 * N * ((double)T * B * 2 * nl + (double)O * B * 2 * nl) + 4.0 * (double)wd_u32,
                (double)O * T * B * 2 * nl * N);
}

// --------------------------------------------------------------- copies
__global__ void gather_rows_kernel(u64 *out, const u64 *in, u32 nrows, size_t in_row_stride_words, u32 logn) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nrows * N) return;
    size_t r = idx >> logn;
    out[idx] = in[r * in_row_stride_words + (idx & (N - 1))];
}

// out[r] = in[r * stride_rows] (rows of N words)
void gather_rows(Ctx *c, u64 *out, const u64 *in, u32 nrows, size_t stride_rows) {
    size_t total = (size_t)nrows * c->N;
    if (!total) return;
    prof_begin(c);
    gather_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, in, nrows, stride_rows * c->N,
                                                                              c->logn);
    note_launch(c, "gather_rows");
}

// --------------------------------------------------------------- stack sum
// out[r][n] = (accumulate ? out[r][n] : 0) + sum_s a[s][r][n], 128-bit lazy
__global__ void sum_stack_kernel(u64 *out, const u64 *__restrict__ a, size_t stride_words, u32 S, u32 nrows,
                                 u32 logn, u32 period, u32 lp, u32 pbase, int accumulate, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nrows * N) return;
    const u32 r = (u32)(idx >> logn);
    const PrimeDev &P = pd[map_prime(r, period, lp, pbase)];
    Acc128 acc = {accumulate ? out[idx] : 0, 0};
    for (u32 s = 0; s < S; ++s) {
        u64 v = a[s * stride_words + idx];
        u64 lo = acc.lo + v;
        acc.hi += lo < v;
        acc.lo = lo;
    }
    out[idx] = reduce128(acc.lo, acc.hi, P);
}

void sum_stack(Ctx *c, u64 *out, const u64 *a, size_t stride_words, u32 S, u32 nrows, u32 period, u32 lp, u32 pbase,
               int accumulate) {
    size_t total = (size_t)nrows * c->N;
    if (!total) return;
    prof_begin(c);
    sum_stack_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(out, a, stride_words, S, nrows, c->logn,
                                                                            period, lp, pbase, accumulate, c->pdev);
    note_launch(c, "sum_stack", 8.0 * total * (S + 1 + (accumulate ? 1 : 0)));
}
