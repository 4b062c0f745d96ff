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
                                                  int accumulate, size_t pt_ostride,
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
    const u32 l = blockIdx.z;
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

void mac(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O, u32 T, u32 B,
         u32 lp, u32 lpq, u32 pbase, int accumulate, size_t pt_ostride) {
    if (!pt_ostride) pt_ostride = (size_t)T * lp * c->N;
    // pt [O][T][lp][N]; x [T] blocks of [B][2][lp][N] at x_tstride; out [O] blocks at out_ostride.
    // Limb l < lpq uses data prime l, limb l >= lpq special prime pbase + l - lpq.
    if (lpq == ~0u) lpq = lp;
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
        dim3 grid((BK + bkc - 1) / bkc, c->N / NT, lp);
        const u64 *ptc = pt + (size_t)o0 * pt_ostride;
        u64 *outc = out + (size_t)o0 * out_ostride;
        prof_begin(c);
#define MAC_LAUNCH(OM, OS)                                                                                        \
    mac_kernel<OM, OS><<<grid, 256, smem, c->stream>>>(outc, x, ptc, oc, T, BK, lp, c->logn, x_tstride, out_ostride, \
                                                       ntlog, tc, lpq, pbase, accumulate, pt_ostride, c->pdev)
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
        note_launch(c, "mac", 8.0 * c->N * ((double)oc * T * lp + (double)T * B * 2 * lp + (double)oc * B * 2 * lp),
                    (double)oc * T * B * 2 * lp * c->N);
    }
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
