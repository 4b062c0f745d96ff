// keyswitch.cu -- hybrid key switching (Han & Ki 2020) and rescale kernels.
//
//   ModUp:   per digit j (consecutive alpha limbs of q_0..q_{lp-1}), fast base
//            conversion (Bajard et al. 2016 / Halevi-Polyakov-Shoup 2018, no
//            correction) of the digit's coefficients to every other limb of
//            Q_l u P, fused with that limb's forward NTT; the digit's own limbs
//            are copied in evaluation form.
//   inner:   acc_k[t] = sum_j D_j[t] (o) ksk_j,k[t] over Q_l u P, 128-bit lazy,
//            with the Galois automorphism applied while loading D (hoisting).
//   ModDown: out_i = (acc_i - BConv_{P->q_i}([acc]_P)) * P^{-1} mod q_i, the
//            conversion, its forward NTT and the combination fused per limb,
//            plus an optional addend (sigma_g(c0) for rotations, d0/d1 for
//            relinearisation).
//   Rescale: c'_i = (c_i - [c_top]_centred) * q_top^{-1} mod q_i, fused the same way.
#include "keyswitch.cuh"
#include "ntt_block.cuh"

// ModUp rows that need a conversion, fused with their forward NTT: row r of the list is
// (offset << 8 | prime) with offset = (b*beta + j)*E + t, t outside digit j.  The CTA (or
// 2-CTA cluster) converts digit j of ciphertext b (coefficient form in xc) to q_t in shared
// memory -- the same base conversion as modup_kernel -- transforms it and writes D.
template <int SPLIT>
__global__ void __launch_bounds__(NTT_MAX_THREADS) modup_ntt_kernel(u64 *D, const u64 *__restrict__ xc, RowSet rs,
                                                         u32 lp, u32 K, u32 alpha, u32 beta, int logn,
                                                         const u64 *__restrict__ tab,
                                                         const u64 *__restrict__ tw_all,
                                                         const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    const Part pt = ntt_part<SPLIT>(logn);
    const u32 v = rs.list[part_row<SPLIT>()];
    const u32 off = v >> 8, prime = v & 0xff;
    const u32 E = lp + K;
    const u32 t = off % E, bj = off / E;
    const u32 j = bj % beta, b = bj / beta;
    const u32 lo = j * alpha;
    const u32 hi = lo + alpha < lp ? lo + alpha : lp;
    const u32 nd = hi - lo;
    const PrimeDev P = pd[prime];
    const u64 *tj = tab + (size_t)j * (2 * alpha + alpha * E);
    const u64 *xb = xc + ((size_t)b * lp + lo) * N;
    if (nd == 1) {
        // single-limb digit: reduce each coefficient (< q_j) mod q_t -- nothing to do when
        // q_j < q_t, one conditional subtraction when q_j < 2 q_t; 16-byte loads, four in flight
        const u64 qj = pd[lo].q;
        const int mode = qj <= P.q ? 0 : qj < 2 * P.q ? 1 : 2;
        const ulonglong2 *x2 = reinterpret_cast<const ulonglong2 *>(xb + pt.lo);
        const u32 half = pt.n / 2;
        for (u32 k0 = threadIdx.x; k0 < half; k0 += 4 * blockDim.x) {
            ulonglong2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const u32 k = k0 + u * blockDim.x;
                if (k < half) v[u] = __ldg(x2 + k);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const u32 k = k0 + u * blockDim.x;
                if (k < half) {
                    u64 a = v[u].x, b = v[u].y;
                    if (mode == 1) {
                        a = a >= P.q ? a - P.q : a;
                        b = b >= P.q ? b - P.q : b;
                    } else if (mode == 2) {
                        a = reduce64(a, P);
                        b = reduce64(b, P);
                    }
                    sm[spad(2 * k)] = a;
                    sm[spad(2 * k + 1)] = b;
                }
            }
        }
    }
    for (u32 n = pt.lo + threadIdx.x; nd > 1 && n < pt.lo + pt.n; n += blockDim.x) {
        u64 o;
        {
            Acc128 acc = {0, 0};
            for (u32 i = 0; i < nd; ++i) {
                const u64 y = mul_shoup(xb[(size_t)i * N + n], tj[i], tj[alpha + i], pd[lo + i].q);
                mac128(acc, y, tj[2 * alpha + (size_t)i * E + t]);
            }
            o = redc128(acc.lo, acc.hi, P);
        }
        sm[spad(n - pt.lo)] = o;
    }
    __syncthreads();
    part_ntt_fwd(sm, pt, logn, tw_all + (size_t)prime * 4 * N, P.q);
    block_store(D + (size_t)off * N + pt.lo, sm, pt.n);
}

// The same rows in the two-kernel form (ntt_block.cuh): the base conversion of each converted
// row's digit computed straight into the registers of its outer forward stages (one column per
// thread), written to D; the inner stages then run over the same rows of D in place.
template <int R>
__global__ void __launch_bounds__(NTT2_COLS) modup2_outer_kernel(u64 *D, const u64 *__restrict__ xc, RowSet rs,
                                                                 u32 lp, u32 K, u32 alpha, u32 beta,
                                                                 const u64 *__restrict__ tab,
                                                                 const u64 *__restrict__ tw_all,
                                                                 const PrimeDev *__restrict__ pd) {
    const u32 N = 1024u << R;
    const u32 v = rs.list[blockIdx.x];
    const u32 off = v >> 8, prime = v & 0xff;
    const u32 E = lp + K;
    const u32 t = off % E, bj = off / E;
    const u32 j = bj % beta, b = bj / beta;
    const u32 lo = j * alpha;
    const u32 hi = lo + alpha < lp ? lo + alpha : lp;
    const u32 nd = hi - lo;
    const PrimeDev P = pd[prime];
    const u64 *tj = tab + (size_t)j * (2 * alpha + alpha * E);
    const u64 *xb = xc + ((size_t)b * lp + lo) * N;
    const u32 g = blockIdx.y * NTT2_COLS + threadIdx.x;
    u64 x[1 << R];
    if (nd == 1) {
        // single-limb digit: each coefficient (< q_j) reduced mod q_t
        const u64 qj = pd[lo].q;
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) {
            u64 a = __ldg(xb + g + 1024u * k);
            if (qj > P.q) a = qj < 2 * P.q ? (a >= P.q ? a - P.q : a) : reduce64(a, P);
            x[k] = a;
        }
    } else {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) {
            const u32 n = g + 1024u * k;
            Acc128 acc = {0, 0};
            for (u32 i = 0; i < nd; ++i) {
                const u64 y = mul_shoup(__ldg(xb + (size_t)i * N + n), tj[i], tj[alpha + i], pd[lo + i].q);
                mac128(acc, y, tj[2 * alpha + (size_t)i * E + t]);
            }
            x[k] = redc128(acc.lo, acc.hi, P);
        }
    }
    outer_fwd_regs<R>(x, tw_all + (size_t)prime * 4 * N, P.q);
    u64 *drow = D + (size_t)off * N + g;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) drow[1024u * k] = x[k];
}

// the digits' own rows of D, copied from the evaluation-form input: D[b][j][t] = xe[b][t], t in digit j
__global__ void modup_own_kernel(u64 *D, const u64 *__restrict__ xe, size_t xe_bstride, u32 lp, u32 K, u32 alpha,
                                 u32 beta, int logn) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 t = blockIdx.y, b = blockIdx.z;
    if (n >= N || t >= lp) return;
    const u32 j = t / alpha, E = lp + K;
    D[(((size_t)b * beta + j) * E + t) * N + n] = xe[(size_t)b * xe_bstride + (size_t)t * N + n];
}

// acc [S][B][2][E][N] = sum_j sigma_g(D_j) (o) key_j; with padd: + P * (padd0, padd1) on the data
// limbs (padd[b] at b * padd_bstride words, polynomial k at k * lp * N; pq: [P]_{q_t} and Shoup pairs)
__global__ void ks_inner_kernel(u64 *acc, const u64 *__restrict__ D, KeyList kl, u32 B, u32 beta, u32 lp, u32 K,
                                u32 L1, int logn, const PrimeDev *__restrict__ pd, const u64 *__restrict__ padd,
                                size_t padd_bstride, const u64 *__restrict__ pq) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u32 t = blockIdx.y;
    const u32 s = blockIdx.z / B, b = blockIdx.z % B;
    const u32 E = lp + K;
    const u32 pt = t < lp ? t : L1 + (t - lp);
    const u32 g = kl.g[s];
    const u64 *key = kl.key[s];
    const u32 src = g == 1 ? n : galois_src(n, g, logn);
    const size_t kstride = (size_t)(L1 + K) * N;
    Acc128 a0 = {0, 0}, a1 = {0, 0};
    const u64 *Db = D + ((size_t)b * beta * E + t) * N + src;
    for (u32 j = 0; j < beta; ++j) {
        const u64 d = Db[(size_t)j * E * N];
        const u64 *kj = key + (size_t)j * 2 * kstride + (size_t)pt * N + n;
        mac128(a0, d, __ldg(kj));
        mac128(a1, d, __ldg(kj + kstride));
    }
    const PrimeDev &P = pd[pt];
    u64 *o = acc + (((size_t)s * B + b) * 2 * E + t) * N + n;
    u64 r0 = redc128(a0.lo, a0.hi, P), r1 = redc128(a1.lo, a1.hi, P);   // keys are in Montgomery form
    if (padd && t < lp) {
        const u64 *x = padd + (size_t)b * padd_bstride + (size_t)t * N + n;
        r0 = add_mod(r0, mul_shoup(x[0], pq[2 * t], pq[2 * t + 1], P.q), P.q);
        r1 = add_mod(r1, mul_shoup(x[(size_t)lp * N], pq[2 * t], pq[2 * t + 1], P.q), P.q);
    }
    o[0] = r0;
    o[(size_t)E * N] = r1;
}

// Accumulators of a hoisted linear combination, before any ModDown:
//   step with g != 1: A0 = sum_j sigma_g(D_j) (o) ksk_j,0 + P*sigma_g(c0)   (P*x is 0 on special limbs)
//                     A1 = sum_j sigma_g(D_j) (o) ksk_j,1
//   step with g == 1: A = (P*c0, P*c1)
// acc [S][B][2][lp+K][N]; x: the input ciphertexts [B][2][lp][N]; pq: [P]_{q_t} and Shoup pairs.
__global__ void ks_lazy_kernel(u64 *acc, const u64 *__restrict__ D, const u64 *__restrict__ x, KeyList kl,
                               u32 B, u32 beta, u32 lp, u32 K, u32 L1, int logn, const u64 *__restrict__ pq,
                               const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u32 t = blockIdx.y;
    const u32 s = blockIdx.z / B, b = blockIdx.z % B;
    const u32 E = lp + K;
    const u32 pt = t < lp ? t : L1 + (t - lp);
    const PrimeDev &P = pd[pt];
    const u32 g = kl.g[s];
    const u64 *xb = x + (size_t)b * 2 * lp * N;
    u64 *o = acc + (((size_t)s * B + b) * 2 * E + t) * N + n;
    if (g == 1) {
        u64 r0 = 0, r1 = 0;
        if (t < lp) {
            r0 = mul_shoup(xb[(size_t)t * N + n], pq[2 * t], pq[2 * t + 1], P.q);
            r1 = mul_shoup(xb[(size_t)(lp + t) * N + n], pq[2 * t], pq[2 * t + 1], P.q);
        }
        o[0] = r0;
        o[(size_t)E * N] = r1;
        return;
    }
    const u64 *key = kl.key[s];
    const u32 src = galois_src(n, g, logn);
    const size_t kstride = (size_t)(L1 + K) * N;
    Acc128 a0 = {0, 0}, a1 = {0, 0};
    const u64 *Db = D + ((size_t)b * beta * E + t) * N + src;
    for (u32 j = 0; j < beta; ++j) {
        const u64 d = Db[(size_t)j * E * N];
        const u64 *kj = key + (size_t)j * 2 * kstride + (size_t)pt * N + n;
        mac128(a0, d, __ldg(kj));
        mac128(a1, d, __ldg(kj + kstride));
    }
    u64 r0 = redc128(a0.lo, a0.hi, P);   // keys are in Montgomery form
    if (t < lp) r0 = add_mod(r0, mul_shoup(xb[(size_t)t * N + src], pq[2 * t], pq[2 * t + 1], P.q), P.q);
    o[0] = r0;
    o[(size_t)E * N] = redc128(a1.lo, a1.hi, P);
}

// Same accumulators, computed with keys stored pre-permuted: K'_{g,j} = sigma_g^{-1}(K_{g,j}), so
//   A_s = sigma_g(A'_s),  A'_s = sum_j D_j (o) K'_j  (+ P*c0 on poly 0),
// i.e. every thread reads its digits D_j[b][t][n] and c0, c1 once (coalesced) and reuses them
// for all S steps; the permutation is applied on the write: A_s[galois_src(n, g^-1)] = A'_s[n].
// Grid: z = limb; x/y = n-tile and ciphertext group, n-tile fastest (order 0: the scattered
// writes of one limb merge in L2) or ciphertext group fastest (order 1: consecutive CTAs
// read the same key slice).  Each thread handles BT ciphertexts of one coefficient so that
// every key word it loads serves BT products; MAXD >= the number of digits.
// Three CTAs per SM (24 warps: the 64-bit multiply chains need the latency hiding) except
// for four ciphertexts of eight digits per thread, which needs the registers of two.
template <int BT, int MAXD>
__global__ void __launch_bounds__(256, (BT == 4 && MAXD == 8) ? 2 : 3) ks_lazy_perm_kernel(u64 *__restrict__ acc, const u64 *__restrict__ D,
                                                            const u64 *__restrict__ x, KeyList kl, u32 S, u32 B,
                                                            u32 beta, u32 lp, u32 K, u32 L1, int logn, int order,
                                                            const u64 *__restrict__ pq,
                                                            const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 ntile = order ? blockIdx.y : blockIdx.x, bgrp = order ? blockIdx.x : blockIdx.y;
    const u32 n = ntile * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u32 b0 = bgrp * BT, t = blockIdx.z;
    const u32 E = lp + K;
    const u32 pt = t < lp ? t : L1 + (t - lp);
    const PrimeDev P = pd[pt];
    u64 d[BT][MAXD];
    u64 pc0[BT], pc1[BT];   // P*c0, P*c1 on data limbs
#pragma unroll
    for (int u = 0; u < BT; ++u) {
        const u32 b = b0 + u < B ? b0 + u : B - 1;   // clamp: duplicates are computed but not stored
        // D is null when every step of the launch is the identity (no digit is read then)
        const u64 *Db = D ? D + ((size_t)b * beta * E + t) * N + n : nullptr;
#pragma unroll
        for (u32 j = 0; j < MAXD; ++j) d[u][j] = (Db && j < beta) ? Db[(size_t)j * E * N] : 0;
        const u64 *xb = x + (size_t)b * 2 * lp * N;
        pc0[u] = pc1[u] = 0;
        if (t < lp) {
            pc0[u] = mul_shoup(xb[(size_t)t * N + n], pq[2 * t], pq[2 * t + 1], P.q);
            pc1[u] = mul_shoup(xb[(size_t)(lp + t) * N + n], pq[2 * t], pq[2 * t + 1], P.q);
        }
    }
    const size_t kstride = (size_t)(L1 + K) * N;
    // the key words of step s+1 are copied into shared memory (cp.async) while step s
    // computes: buffer layout [2][2 polys][MAXD][256 threads], each thread its own slots
    extern __shared__ u64 ksm[];
    auto issue = [&](u32 s, u32 buf) {
        if (kl.g[s] != 1) {
            const u64 *key = kl.keyp[s] + (size_t)pt * N + n;
#pragma unroll
            for (u32 j = 0; j < MAXD; ++j)
                if (j < beta) {
                    cp_async8(ksm + ((buf * 2 + 0) * MAXD + j) * 256 + threadIdx.x, key + (size_t)j * 2 * kstride);
                    cp_async8(ksm + ((buf * 2 + 1) * MAXD + j) * 256 + threadIdx.x,
                              key + (size_t)j * 2 * kstride + kstride);
                }
        }
        cp_commit();
    };
    issue(0, 0);
    for (u32 s = 0; s < S; ++s) {
        const u32 g = kl.g[s];
        if (s + 1 < S)
            issue(s + 1, (s + 1) & 1);
        else
            cp_commit();
        cp_wait<1>();   // the copies of step s have landed
        const u64 *k0 = ksm + ((s & 1) * 2 + 0) * MAXD * 256 + threadIdx.x;
        const u64 *k1 = ksm + ((s & 1) * 2 + 1) * MAXD * 256 + threadIdx.x;
        const u32 dst = g == 1 ? n : galois_src(n, kl.ginv[s], logn);
        u64 *os = acc + (((size_t)s * B + b0) * 2 * E + t) * N;   // step s, ciphertext b0
#pragma unroll
        for (int u = 0; u < BT; ++u) {
            if (b0 + u >= B) break;
            u64 *o = os + (size_t)u * 2 * E * N;
            if (g == 1) {
                o[n] = pc0[u];
                o[(size_t)E * N + n] = pc1[u];
                continue;
            }
            Acc128 a0 = {0, 0}, a1 = {0, 0};
#pragma unroll
            for (u32 j = 0; j < MAXD; ++j) {
                if (j < beta) {
                    mac128(a0, d[u][j], k0[j * 256]);
                    mac128(a1, d[u][j], k1[j * 256]);
                }
            }
            // keys are in Montgomery form: one Montgomery reduction per sum
            o[dst] = add_mod(redc128(a0.lo, a0.hi, P), pc0[u], P.q);
            o[(size_t)E * N + dst] = redc128(a1.lo, a1.hi, P);
        }
    }
}

// A weighted hoisted linear combination accumulated in one pass, with the digits gathered at each
// step's Galois permutation (the addressing of ks_inner_kernel) instead of one accumulator per
// step written out and summed by a second kernel:
//   Z[b] (+)= sum_{s<S} sum_{i<CH} w[s*CH + i] (.) A_s(X_{i*B+b})
// with A_s(X) = (sum_j sigma_g(D_j) (.) ksk_{g,j,0} + P*sigma_g(c0),  sum_j sigma_g(D_j) (.) ksk_{g,j,1})
// over Q_l u P (A_s = (P*c0, P*c1) for g = 1) -- the accumulators of ks_lazy_kernel, same values.
// Z [B][2][E][N]; w [S*CH][E][N].  Each step's key sum is reduced (REDC) and multiplied by its
// weight into a 128-bit sum (folded every 64 terms).  One thread per coefficient of one limb for BT
// ciphertexts, both polynomials; grid (n-tiles, ciphertext groups, limbs), n-tiles fastest, so the
// digit rows of a group stay in L2 while their tiles are gathered.  For the combinations of one
// channel over many ciphertexts ks_comb_lazy_kernel (weights folded into the keys) takes over.
// MAXD > 0: at most MAXD digits, unrolled; MAXD = 0: any digit count.
template <int BT, int MAXD>
__global__ void __launch_bounds__(256, BT == 2 ? 3 : 2) ks_comb_kernel(u64 *__restrict__ Z, const u64 *__restrict__ D,
                                                      const u64 *__restrict__ x, KeyList kl, u32 S, u32 CH, u32 B,
                                                      u32 beta, u32 lp, u32 K, u32 L1, int logn,
                                                      const u64 *__restrict__ w, int accumulate,
                                                      const u64 *__restrict__ pq, const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 t = blockIdx.z;
    const u32 E = lp + K;
    const u32 pt = t < lp ? t : L1 + (t - lp);
    const PrimeDev P = pd[pt];
    const size_t kstride = (size_t)(L1 + K) * N;
    const u32 c0 = blockIdx.y * BT;   // ciphertexts c0 .. c0 + BT - 1 of every channel
    if (n >= N) return;
    Acc128 zw[BT][2];
#pragma unroll
    for (int u = 0; u < BT; ++u) zw[u][0] = zw[u][1] = Acc128{0, 0};
    u32 terms = 0;
    for (u32 s = 0; s < S; ++s) {
        const u32 g = kl.g[s];
        const u32 src = g == 1 ? n : galois_src(n, g, logn);
        const u64 *kp = g == 1 ? nullptr : kl.key[s] + (size_t)pt * N + n;
        for (u32 i = 0; i < CH; ++i) {
            u64 a[BT][2];
            if (g == 1) {
#pragma unroll
                for (int u = 0; u < BT; ++u) {
                    const u32 bb = c0 + u < B ? c0 + u : B - 1;   // clamp: duplicates are not stored
                    const u64 *xb = x + (size_t)(i * B + bb) * 2 * lp * N;
                    a[u][0] = t < lp ? mul_shoup(xb[(size_t)t * N + n], pq[2 * t], pq[2 * t + 1], P.q) : 0;
                    a[u][1] = t < lp ? mul_shoup(xb[(size_t)(lp + t) * N + n], pq[2 * t], pq[2 * t + 1], P.q) : 0;
                }
            } else {
                Acc128 s0[BT], s1[BT];
                size_t db[BT];   // word offset of each ciphertext's digit 0 at the gathered coefficient
#pragma unroll
                for (int u = 0; u < BT; ++u) {
                    const u32 bb = c0 + u < B ? c0 + u : B - 1;
                    db[u] = ((size_t)(i * B + bb) * beta * E + t) * N + src;
                    s0[u] = s1[u] = Acc128{0, 0};
                }
                // each key word is loaded once per channel and serves the BT ciphertexts
                auto digit = [&](u32 j) {
                    const u64 k0 = __ldg(kp + (size_t)j * 2 * kstride), k1 = __ldg(kp + (size_t)j * 2 * kstride + kstride);
#pragma unroll
                    for (int u = 0; u < BT; ++u) {
                        const u64 d = D[db[u] + (size_t)j * E * N];
                        mac128(s0[u], d, k0);
                        mac128(s1[u], d, k1);
                    }
                };
                if constexpr (MAXD > 0) {
#pragma unroll
                    for (int j = 0; j < MAXD; ++j)
                        if (j < (int)beta) digit((u32)j);
                } else {
                    for (u32 j = 0; j < beta; ++j) digit(j);
                }
#pragma unroll
                for (int u = 0; u < BT; ++u) {
                    const u32 bb = c0 + u < B ? c0 + u : B - 1;
                    const u64 *xb = x + (size_t)(i * B + bb) * 2 * lp * N;
                    u64 r0 = redc128(s0[u].lo, s0[u].hi, P);   // keys are in Montgomery form
                    if (t < lp)
                        r0 = add_mod(r0, mul_shoup(xb[(size_t)t * N + src], pq[2 * t], pq[2 * t + 1], P.q), P.q);
                    a[u][0] = r0;
                    a[u][1] = redc128(s1[u].lo, s1[u].hi, P);
                }
            }
            const u64 wv = __ldg(w + ((size_t)(s * CH + i) * E + t) * N + n);
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                mac128(zw[u][0], a[u][0], wv);
                mac128(zw[u][1], a[u][1], wv);
            }
            if (++terms == 64) {   // products < 2^122: fold before the 128-bit sums can overflow
                terms = 0;
#pragma unroll
                for (int u = 0; u < BT; ++u)
#pragma unroll
                    for (int k = 0; k < 2; ++k) zw[u][k] = Acc128{reduce128(zw[u][k].lo, zw[u][k].hi, P), 0};
            }
        }
    }
    const size_t zct = (size_t)2 * E * N;   // one output ciphertext over Q_l u P
#pragma unroll
    for (int u = 0; u < BT; ++u) {
        if (c0 + u >= B) break;
        u64 *zo = Z + (size_t)(c0 + u) * zct + (size_t)t * N + n;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            u64 v = reduce128(zw[u][k].lo, zw[u][k].hi, P);
            if (accumulate) v = add_mod(v, zo[(size_t)k * E * N], P.q);
            zo[(size_t)k * E * N] = v;
        }
    }
}

// The same combinations with one lazy 128-bit sum per output polynomial and one reduction at
// the end, for plain sums and for single-output weighted sums of one channel whose weights were
// folded into the keys beforehand (ks_fold_kernel):
//   poly 0: Z[c] (+)= REDC( sum_s [ sum_j sigma_s(D_j) (.) K'_{s,j,0} + sigma_s(c0) (.) P'_s ] )
//   poly 1: Z[c] (+)= REDC( sum_s   sum_j sigma_s(D_j) (.) K'_{s,j,1} )
// (an identity step adds c0 (.) P'_s and c1 (.) P'_s), every operand K', P' carrying a factor
// 2^64 that the one Montgomery reduction of the reduced sum removes:
//   plain:    K' = the Montgomery keys,   P'_s = [P 2^64]_{q_t};
//   weighted: K' = K~ (.) w_s (K~ the Montgomery key),  P'_s = [P 2^64]_{q_t} (.) w_s.
// These are the residues of ks_comb_kernel, summed in another order: identical results, without a
// reduction and a Shoup product per step.  Keys of step s at kl.key[s] + j*2*kst + k*kst +
// row*N, row = t on a data limb, krow_sp + (t - lp) on a special one; pw [S][lp][N] (weighted) or
// null (plain: pmont [2*t] = [P 2^64]_{q_t}).  Grid as ks_comb_kernel, one ciphertext each of BT.
template <int BT, int MAXD>
__global__ void __launch_bounds__(256, BT == 2 ? 3 : 2) ks_comb_lazy_kernel(
    u64 *__restrict__ Z, const u64 *__restrict__ D, const u64 *__restrict__ x, KeyList kl, u32 S, u32 nb, u32 beta,
    u32 lp, u32 K, u32 L1, u32 krow_sp, size_t kst, const u64 *__restrict__ pw, const u64 *__restrict__ pmont,
    int accumulate, int logn, const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 t = blockIdx.z;
    const u32 E = lp + K;
    const PrimeDev P = pd[t < lp ? t : L1 + (t - lp)];
    const u32 krow = t < lp ? t : krow_sp + (t - lp);
    const u32 c0 = blockIdx.y * BT;
    if (n >= N) return;
    Acc128 z[BT][2];
#pragma unroll
    for (int u = 0; u < BT; ++u) z[u][0] = z[u][1] = Acc128{0, 0};
    const u32 per = (MAXD > 0 ? (u32)MAXD : beta) + 1;   // products one step adds to a sum, at most
    u32 terms = 0;
    for (u32 s = 0; s < S; ++s) {
        if (terms + per > 63) {   // products < 2^122: fold before a 128-bit sum could overflow
#pragma unroll
            for (int u = 0; u < BT; ++u)
#pragma unroll
                for (int k = 0; k < 2; ++k) z[u][k] = Acc128{reduce128(z[u][k].lo, z[u][k].hi, P), 0};
            terms = 0;
        }
        terms += per;
        const u32 g = kl.g[s];
        const u32 src = g == 1 ? n : galois_src(n, g, logn);
        const u64 cw = t < lp ? (pw ? pw[((size_t)s * lp + t) * N + n] : pmont[2 * t]) : 0;
        if (g == 1) {
            if (t < lp) {
#pragma unroll
                for (int u = 0; u < BT; ++u) {
                    const u32 bb = c0 + u < nb ? c0 + u : nb - 1;   // clamp: duplicates are not stored
                    const u64 *xb = x + (size_t)bb * 2 * lp * N;
                    mac128(z[u][0], xb[(size_t)t * N + n], cw);
                    mac128(z[u][1], xb[(size_t)(lp + t) * N + n], cw);
                }
            }
            continue;
        }
        const u64 *kp = kl.key[s] + (size_t)krow * N + n;
        size_t db[BT];   // word offset of each ciphertext's digit 0 at the gathered coefficient
#pragma unroll
        for (int u = 0; u < BT; ++u) {
            const u32 bb = c0 + u < nb ? c0 + u : nb - 1;   // clamp: duplicates are not stored
            db[u] = ((size_t)bb * beta * E + t) * N + src;
        }
        // each key word is loaded once and serves the BT ciphertexts
        if constexpr (MAXD > 0) {
#pragma unroll
            for (int j = 0; j < MAXD; ++j)
                if (j < (int)beta) {
                    const u64 k0 = __ldg(kp + (size_t)j * 2 * kst), k1 = __ldg(kp + (size_t)j * 2 * kst + kst);
#pragma unroll
                    for (int u = 0; u < BT; ++u) {
                        const u64 d = D[db[u] + (size_t)j * E * N];
                        mac128(z[u][0], d, k0);
                        mac128(z[u][1], d, k1);
                    }
                }
        } else {
            for (u32 j = 0; j < beta; ++j) {
                const u64 k0 = __ldg(kp + (size_t)j * 2 * kst), k1 = __ldg(kp + (size_t)j * 2 * kst + kst);
#pragma unroll
                for (int u = 0; u < BT; ++u) {
                    const u64 d = D[db[u] + (size_t)j * E * N];
                    mac128(z[u][0], d, k0);
                    mac128(z[u][1], d, k1);
                }
            }
        }
        if (t < lp) {
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const u32 bb = c0 + u < nb ? c0 + u : nb - 1;
                mac128(z[u][0], x[(size_t)bb * 2 * lp * N + (size_t)t * N + src], cw);
            }
        }
    }
    const size_t zct = (size_t)2 * E * N;   // one output ciphertext over Q_l u P
#pragma unroll
    for (int u = 0; u < BT; ++u) {
        if (c0 + u >= nb) break;
        u64 *zo = Z + (size_t)(c0 + u) * zct + (size_t)t * N + n;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            u64 v = redc128(reduce128(z[u][k].lo, z[u][k].hi, P), 0, P);   // the sum times 2^-64
            if (accumulate) v = add_mod(v, zo[(size_t)k * E * N], P.q);
            zo[(size_t)k * E * N] = v;
        }
    }
}

// The operands of a single-output weighted combination of one channel for ks_comb_lazy_kernel,
// with the weights w [S][E][N] (over Q_l u P) folded in:
//   F [S][beta][2][E][N]: K' (.) w_s of every key-switched step (K' the Montgomery key);
//   pw [S][lp][N]: [P 2^64]_{q_t} (.) w_s on the data limbs.
// Grid (n-tiles, E, S).
__global__ void ks_fold_kernel(u64 *__restrict__ F, u64 *__restrict__ pw, KeyList kl, const u64 *__restrict__ w,
                               u32 beta, u32 lp, u32 K, u32 L1, int logn, const u64 *__restrict__ pmont,
                               const PrimeDev *__restrict__ pd) {
    const u32 N = 1u << logn;
    const u32 n = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 t = blockIdx.y, s = blockIdx.z;
    if (n >= N) return;
    const u32 E = lp + K;
    const u32 pt = t < lp ? t : L1 + (t - lp);
    const PrimeDev P = pd[pt];
    const u64 wv = w[((size_t)s * E + t) * N + n];
    if (kl.g[s] != 1) {
        const size_t kstride = (size_t)(L1 + K) * N;
        const u64 *key = kl.key[s] + (size_t)pt * N + n;
        u64 *f = F + ((size_t)s * beta * 2 * E + t) * N + n;
        for (u32 j = 0; j < beta; ++j)
#pragma unroll
            for (u32 k = 0; k < 2; ++k)
                f[((size_t)j * 2 + k) * E * N] = mul_mod(__ldg(key + (size_t)j * 2 * kstride + k * kstride), wv, P);
    }
    if (t < lp) pw[((size_t)s * lp + t) * N + n] = mul_shoup(wv, pmont[2 * t], pmont[2 * t + 1], P.q);
}

// Division by the dropped basis D of the accumulators acc [S][B][2][lp+K][N]: D is
// the KD rows starting at row dbase (dbase = lp: the special primes, ModDown;
// dbase = lp-1: the top data prime and the special primes, ModDown and rescale in
// one).  Output limb i < lpo: (acc_i - BConv_{D->q_i}) * D^{-1}, plus the addend.
template <int SPLIT>
__global__ void __launch_bounds__(NTT_MAX_THREADS) moddown_kernel(u64 *out, const u64 *__restrict__ acc,
                                                       const u64 *__restrict__ addend, size_t addend_bstride,
                                                       u32 add_mask, KeyList kl, u32 B, u32 lp, u32 K, u32 L1,
                                                       u32 dbase, u32 KD, u32 lpo, int logn,
                                                       const u64 *__restrict__ mdtab,
                                                       const u64 *__restrict__ tw_all,
                                                       const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    const Part pt = ntt_part<SPLIT>(logn);
    const u32 i = part_row<SPLIT>(), k = blockIdx.y;
    const u32 s = blockIdx.z / B, b = blockIdx.z % B;
    const u32 E = lp + K;
    const PrimeDev P = pd[i];
    const u64 *ab = acc + (((size_t)s * B + b) * 2 + k) * E * N;
    const bool add = addend && ((add_mask >> k) & 1);
    const u64 *adb = add ? addend + (size_t)b * addend_bstride + ((size_t)k * lpo + i) * N : nullptr;
    if (threadIdx.x == 0) {
        // the rows the combination reads after the NTT are pulled into L2 meanwhile (bulk prefetch)
        l2_prefetch_bulk(ab + (size_t)i * N + pt.lo, pt.n * 8);
        if (add) l2_prefetch_bulk(adb, N * 8);
    }
    // mdtab: dhinv[KD], dhinv_s[KD], dhmod[KD][L1], Dinv[L1], Dinv_s[L1]
    // base conversion of two coefficients per thread and iteration (16-byte loads)
    const u32 half = pt.n / 2;
    for (u32 k2 = threadIdx.x; k2 < half; k2 += blockDim.x) {
        const u32 n = pt.lo + 2 * k2;
        u64 v0, v1;
        if (KD == 1) {
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ab + (size_t)dbase * N + n);
            v0 = reduce64(x.x, P);
            v1 = reduce64(x.y, P);
        } else {
            Acc128 a0 = {0, 0}, a1 = {0, 0};
            for (u32 kk = 0; kk < KD; ++kk) {
                const u32 row = dbase + kk;
                const PrimeDev &Pk = pd[row < lp ? row : L1 + (row - lp)];
                const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ab + (size_t)row * N + n);
                const u64 hm = mdtab[2 * KD + (size_t)kk * L1 + i];   // Montgomery form
                mac128(a0, mul_shoup(x.x, mdtab[kk], mdtab[KD + kk], Pk.q), hm);
                mac128(a1, mul_shoup(x.y, mdtab[kk], mdtab[KD + kk], Pk.q), hm);
            }
            v0 = redc128(a0.lo, a0.hi, P);
            v1 = redc128(a1.lo, a1.hi, P);
        }
        sm[spad(2 * k2)] = v0;
        sm[spad(2 * k2 + 1)] = v1;
    }
    __syncthreads();
    part_ntt_fwd(sm, pt, logn, tw_all + (size_t)i * 4 * N, P.q);
    const u64 pinv = mdtab[2 * KD + (size_t)KD * L1 + i];
    const u64 pinvs = mdtab[2 * KD + (size_t)KD * L1 + L1 + i];
    const u32 g = kl.g[s];
    u64 *ob = out + ((((size_t)s * B + b) * 2 + k) * lpo + i) * N;
    for (u32 k2 = threadIdx.x; k2 < half; k2 += blockDim.x) {
        const u32 n = pt.lo + 2 * k2;
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ab + (size_t)i * N + n);
        u64 o0 = mul_shoup(sub_mod(x.x, sm[spad(2 * k2)], P.q), pinv, pinvs, P.q);
        u64 o1 = mul_shoup(sub_mod(x.y, sm[spad(2 * k2 + 1)], P.q), pinv, pinvs, P.q);
        if (add) {
            o0 = add_mod(o0, adb[g == 1 ? n : galois_src(n, g, logn)], P.q);
            o1 = add_mod(o1, adb[g == 1 ? n + 1 : galois_src(n + 1, g, logn)], P.q);
        }
        ulonglong2 r;
        r.x = o0;
        r.y = o1;
        *reinterpret_cast<ulonglong2 *>(ob + n) = r;
    }
}

// ModDown (or ModDown + rescale) in the two-kernel form.  Rows of the output: r =
// ((s*B + b)*2 + k)*lpo + i.  The outer launch converts the dropped rows of acc (D -> q_i) straight
// into the registers of the row's outer forward stages and writes them to the output row; the
// inner launch runs the inner stages of each 1024-coefficient block in place and combines:
// out = (acc_i - conv) * D^-1 (+ the addend gathered by sigma_g), as moddown_kernel does.
template <int R>
__global__ void __launch_bounds__(NTT2_COLS) moddown2_outer_kernel(u64 *out, const u64 *__restrict__ acc, u32 lp,
                                                                   u32 K, u32 L1, u32 dbase, u32 KD, u32 lpo,
                                                                   const u64 *__restrict__ mdtab,
                                                                   const u64 *__restrict__ tw_all,
                                                                   const PrimeDev *__restrict__ pd) {
    const u32 N = 1024u << R;
    const u32 r = blockIdx.x, i = r % lpo, sbk = r / lpo;
    const u32 E = lp + K;
    const PrimeDev P = pd[i];
    const u64 *ab = acc + (size_t)sbk * E * N;
    const u32 g = blockIdx.y * NTT2_COLS + threadIdx.x;
    u64 x[1 << R];
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        const u32 n = g + 1024u * k;
        if (KD == 1) {
            x[k] = reduce64(ab[(size_t)dbase * N + n], P);
        } else {
            Acc128 a = {0, 0};
            for (u32 kk = 0; kk < KD; ++kk) {
                const u32 row = dbase + kk;
                const PrimeDev &Pk = pd[row < lp ? row : L1 + (row - lp)];
                const u64 hm = mdtab[2 * KD + (size_t)kk * L1 + i];   // Montgomery form
                mac128(a, mul_shoup(ab[(size_t)row * N + n], mdtab[kk], mdtab[KD + kk], Pk.q), hm);
            }
            x[k] = redc128(a.lo, a.hi, P);
        }
    }
    outer_fwd_regs<R>(x, tw_all + (size_t)i * 4 * N, P.q);
    u64 *orow = out + (size_t)r * N + g;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) orow[1024u * k] = x[k];
}

__global__ void __launch_bounds__(NTT2_INNER_THREADS) moddown2_inner_kernel(
    u64 *out, const u64 *__restrict__ acc, const u64 *__restrict__ addend, size_t addend_bstride, u32 add_mask,
    KeyList kl, u32 B, u32 lp, u32 K, u32 L1, u32 KD, u32 lpo, int logn, const u64 *__restrict__ mdtab,
    const u64 *__restrict__ tw_all, const PrimeDev *__restrict__ pd) {
    __shared__ u64 sm[1024 + 1024 / 16];
    const u32 N = 1u << logn;
    const u32 r = blockIdx.x, i = r % lpo, sbk = r / lpo;
    const u32 k = sbk & 1, sb = sbk >> 1, s = sb / B, b = sb % B;
    const u32 E = lp + K;
    const PrimeDev P = pd[i];
    const u32 goff = 1024u * blockIdx.y;
    u64 *ob = out + (size_t)r * N;
    block_load(sm, ob + goff, 1024);
    inner_fwd_block(sm, logn, tw_all + (size_t)i * 4 * N, P.q, goff);
    const u64 pinv = mdtab[2 * KD + (size_t)KD * L1 + i];
    const u64 pinvs = mdtab[2 * KD + (size_t)KD * L1 + L1 + i];
    const u64 *ai = acc + (size_t)sbk * E * N + (size_t)i * N;
    const bool add = addend && ((add_mask >> k) & 1);
    const u64 *adb = add ? addend + (size_t)b * addend_bstride + ((size_t)k * lpo + i) * N : nullptr;
    const u32 g = kl.g[s];
    for (u32 k2 = threadIdx.x; k2 < 512; k2 += blockDim.x) {
        const u32 n = goff + 2 * k2;
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ai + n);
        u64 o0 = mul_shoup(sub_mod(x.x, sm[spad(2 * k2)], P.q), pinv, pinvs, P.q);
        u64 o1 = mul_shoup(sub_mod(x.y, sm[spad(2 * k2 + 1)], P.q), pinv, pinvs, P.q);
        if (add) {
            o0 = add_mod(o0, adb[g == 1 ? n : galois_src(n, g, logn)], P.q);
            o1 = add_mod(o1, adb[g == 1 ? n + 1 : galois_src(n + 1, g, logn)], P.q);
        }
        ulonglong2 o;
        o.x = o0;
        o.y = o1;
        *reinterpret_cast<ulonglong2 *>(ob + n) = o;
    }
}

// Rescale in the two-kernel form: rows r = (b*2 + k)*(lp-1) + i of the output; the outer launch
// reduces the centred top limb (coefficient form, top) mod q_i into the outer stages, the inner
// one finishes the NTT and combines out = (in_i - that) * q_top^-1.
template <int R>
__global__ void __launch_bounds__(NTT2_COLS) rescale2_outer_kernel(u64 *out, const u64 *__restrict__ top, u32 lp,
                                                                   const u64 *__restrict__ tw_all,
                                                                   const PrimeDev *__restrict__ pd) {
    const u32 N = 1024u << R;
    const u32 r = blockIdx.x, i = r % (lp - 1), bk = r / (lp - 1);
    const PrimeDev P = pd[i];
    const u64 qt = pd[lp - 1].q;
    const u64 *tb = top + (size_t)bk * N;
    const u32 g = blockIdx.y * NTT2_COLS + threadIdx.x;
    u64 x[1 << R];
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        const u64 v = tb[g + 1024u * k];
        x[k] = v > qt / 2 ? neg_mod(reduce64(qt - v, P), P.q) : reduce64(v, P);
    }
    outer_fwd_regs<R>(x, tw_all + (size_t)i * 4 * N, P.q);
    u64 *orow = out + (size_t)r * N + g;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) orow[1024u * k] = x[k];
}

__global__ void __launch_bounds__(NTT2_INNER_THREADS) rescale2_inner_kernel(u64 *out, const u64 *__restrict__ in,
                                                                            u32 lp, int logn,
                                                                            const u64 *__restrict__ rtab,
                                                                            const u64 *__restrict__ tw_all,
                                                                            const PrimeDev *__restrict__ pd) {
    __shared__ u64 sm[1024 + 1024 / 16];
    const u32 N = 1u << logn;
    const u32 r = blockIdx.x, i = r % (lp - 1), bk = r / (lp - 1);
    const PrimeDev P = pd[i];
    const u32 goff = 1024u * blockIdx.y;
    u64 *ob = out + (size_t)r * N;
    block_load(sm, ob + goff, 1024);
    inner_fwd_block(sm, logn, tw_all + (size_t)i * 4 * N, P.q, goff);
    const u64 w = rtab[i], ws = rtab[lp - 1 + i];
    const u64 *ib = in + ((size_t)bk * lp + i) * N;
    for (u32 k2 = threadIdx.x; k2 < 512; k2 += blockDim.x) {
        const u32 n = goff + 2 * k2;
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ib + n);
        ulonglong2 o;
        o.x = mul_shoup(sub_mod(x.x, sm[spad(2 * k2)], P.q), w, ws, P.q);
        o.y = mul_shoup(sub_mod(x.y, sm[spad(2 * k2 + 1)], P.q), w, ws, P.q);
        *reinterpret_cast<ulonglong2 *>(ob + n) = o;
    }
}

template <int SPLIT>
__global__ void __launch_bounds__(NTT_MAX_THREADS) rescale_kernel(u64 *out, const u64 *__restrict__ in,
                                                       const u64 *__restrict__ top, u32 lp, int logn,
                                                       const u64 *__restrict__ rtab, const u64 *__restrict__ tw_all,
                                                       const PrimeDev *__restrict__ pd) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    const Part pt = ntt_part<SPLIT>(logn);
    const u32 i = part_row<SPLIT>(), k = blockIdx.y, b = blockIdx.z;
    const PrimeDev P = pd[i];
    const u64 qt = pd[lp - 1].q;
    const u64 *tb = top + ((size_t)b * 2 + k) * N;
    for (u32 n = pt.lo + threadIdx.x; n < pt.lo + pt.n; n += blockDim.x) {
        u64 v = tb[n];
        sm[spad(n - pt.lo)] = v > qt / 2 ? neg_mod(reduce64(qt - v, P), P.q) : reduce64(v, P);
    }
    __syncthreads();
    part_ntt_fwd(sm, pt, logn, tw_all + (size_t)i * 4 * N, P.q);
    const u64 w = rtab[i], ws = rtab[lp - 1 + i];
    const u64 *ib = in + (((size_t)b * 2 + k) * lp + i) * N;
    u64 *ob = out + (((size_t)b * 2 + k) * (lp - 1) + i) * N;
    for (u32 n = pt.lo + threadIdx.x; n < pt.lo + pt.n; n += blockDim.x)
        ob[n] = mul_shoup(sub_mod(ib[n], sm[spad(n - pt.lo)], P.q), w, ws, P.q);
}

// ------------------------------------------------------------------ host
static u64 mulmod_h(u64 a, u64 b, u64 q) { return (u64)((unsigned __int128)a * b % q); }
static u64 powmod_h(u64 a, u64 e, u64 q) {
    u64 r = 1;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_h(r, a, q);
        a = mulmod_h(a, a, q);
        e >>= 1;
    }
    return r;
}
static u64 invmod_h(u64 a, u64 q) { return powmod_h(a, q - 2, q); }
static u64 shoup_h(u64 w, u64 q) { return (u64)(((unsigned __int128)w << 64) / q); }

static void set_big_smem(const void *fn) {
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
}

void keyswitch_init(Ctx *c) {
    // the hoisted accumulation double-buffers its key words: 2 x 2 x MAXD x 256 words of shared memory
    for (const void *f : {(const void *)ks_lazy_perm_kernel<1, 8>, (const void *)ks_lazy_perm_kernel<2, 8>,
                          (const void *)ks_lazy_perm_kernel<4, 8>,
                          (const void *)ks_lazy_perm_kernel<1, 4>, (const void *)ks_lazy_perm_kernel<2, 4>,
                          (const void *)ks_lazy_perm_kernel<4, 4>, (const void *)ks_lazy_perm_kernel<1, 2>,
                          (const void *)ks_lazy_perm_kernel<2, 2>, (const void *)ks_lazy_perm_kernel<4, 2>})
        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    set_big_smem((const void *)modup_ntt_kernel<0>);
    set_big_smem((const void *)modup_ntt_kernel<1>);
    set_big_smem((const void *)moddown_kernel<0>);
    set_big_smem((const void *)moddown_kernel<1>);
    set_big_smem((const void *)rescale_kernel<0>);
    set_big_smem((const void *)rescale_kernel<1>);
}

u32 ks_digits(const Ctx *c, u32 lp) { return (lp + c->alpha - 1) / c->alpha; }

// ModUp constants for level lp: per digit j: qhinv[alpha], qhinv_s[alpha], qhmod[alpha][lp+K]
// (qhmod in Montgomery form: the conversion sum of at most 8 terms is reduced with one REDC)
static const u64 *modup_table(Ctx *c, u32 lp) {
    std::string key = fmt("modup:%u", lp);
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second.p;
    const u32 E = lp + c->K, A = c->alpha, beta = ks_digits(c, lp);
    std::vector<u64> h((size_t)beta * (2 * A + A * E), 0);
    for (u32 j = 0; j < beta; ++j) {
        u32 lo = j * A, hi = std::min(lo + A, lp);
        u64 *tj = h.data() + (size_t)j * (2 * A + A * E);
        for (u32 i = lo; i < hi; ++i) {
            u64 qi = c->primes[i];
            u64 hh = 1;
            for (u32 k = lo; k < hi; ++k)
                if (k != i) hh = mulmod_h(hh, c->primes[k] % qi, qi);
            u64 inv = invmod_h(hh, qi);
            tj[i - lo] = inv;
            tj[A + i - lo] = shoup_h(inv, qi);
            for (u32 t = 0; t < E; ++t) {
                u64 pt = c->primes[t < lp ? t : c->L1 + (t - lp)];
                u64 m = 1;
                for (u32 k = lo; k < hi; ++k)
                    if (k != i) m = mulmod_h(m, c->primes[k] % pt, pt);
                tj[2 * A + (size_t)(i - lo) * E + t] = (u64)(((unsigned __int128)m << 64) % pt);   // Montgomery form
            }
        }
    }
    return c->const_table(key, h);
}

// Division table of a dropped basis D = {d_0..d_{KD-1}} (prime indices dp) onto the data primes:
// dhinv[KD], dhinv_s[KD] ((D/d_k)^{-1} mod d_k), dhmod[KD][L1] ((D/d_k) * 2^64 mod q_i: Montgomery
// form, the conversion sum is reduced with one REDC), Dinv[L1], Dinv_s[L1]
static const u64 *drop_table(Ctx *c, const std::string &key, const std::vector<u32> &dp) {
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second.p;
    const u32 KD = (u32)dp.size(), L1 = c->L1;
    std::vector<u64> h(2 * KD + (size_t)KD * L1 + 2 * L1, 0);
    for (u32 k = 0; k < KD; ++k) {
        u64 pk = c->primes[dp[k]];
        u64 hh = 1;
        for (u32 m = 0; m < KD; ++m)
            if (m != k) hh = mulmod_h(hh, c->primes[dp[m]] % pk, pk);
        h[k] = invmod_h(hh, pk);
        h[KD + k] = shoup_h(h[k], pk);
        for (u32 i = 0; i < L1; ++i) {
            u64 qi = c->primes[i], m2 = 1;
            for (u32 m = 0; m < KD; ++m)
                if (m != k) m2 = mulmod_h(m2, c->primes[dp[m]] % qi, qi);
            h[2 * KD + (size_t)k * L1 + i] = (u64)(((unsigned __int128)m2 << 64) % qi);
        }
    }
    for (u32 i = 0; i < L1; ++i) {
        u64 qi = c->primes[i], D = 1;
        for (u32 k = 0; k < KD; ++k) D = mulmod_h(D, c->primes[dp[k]] % qi, qi);
        u64 inv = D ? invmod_h(D, qi) : 0;   // D = 0 mod q_i only for the dropped data prime itself (never an output)
        h[2 * KD + (size_t)KD * L1 + i] = inv;
        h[2 * KD + (size_t)KD * L1 + L1 + i] = shoup_h(inv, qi);
    }
    return c->const_table(key, h);
}

static const u64 *moddown_table(Ctx *c) {
    std::vector<u32> dp;
    for (u32 k = 0; k < c->K; ++k) dp.push_back(c->L1 + k);
    return drop_table(c, "moddown", dp);
}

static const u64 *moddown_rescale_table(Ctx *c, u32 lp) {
    std::vector<u32> dp{lp - 1};
    for (u32 k = 0; k < c->K; ++k) dp.push_back(c->L1 + k);
    return drop_table(c, fmt("moddown_rs:%u", lp), dp);
}

static const u64 *rescale_table(Ctx *c, u32 lp) {
    std::string key = fmt("rescale:%u", lp);
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second.p;
    std::vector<u64> h(2 * (lp - 1));
    u64 qt = c->primes[lp - 1];
    for (u32 i = 0; i + 1 < lp; ++i) {
        u64 qi = c->primes[i];
        u64 inv = invmod_h(qt % qi, qi);
        h[i] = inv;
        h[lp - 1 + i] = shoup_h(inv, qi);
    }
    return c->const_table(key, h);
}

// D [B][beta][lp+K][N] from x: coefficient copy xc [B][lp][N] and eval rows at xe (+ b*xe_bstride)
void ks_modup(Ctx *c, u64 *D, const u64 *xe, size_t xe_bstride, u32 B, u32 lp) {
    const u32 N = c->N, E = lp + c->K, beta = ks_digits(c, lp);
    if ((size_t)B * beta * E >= (1u << 24)) throw HeError(HE_EINVAL, "ModUp: batch too large for one launch");
    DBuf xc(c, (size_t)B * lp * N);
    // the eval rows in coefficient form, contiguous (and copied to the digits' own rows of D as read)
    const bool own_done = ntt_inverse_from(c, xc.p, xe, xe_bstride, B, lp, D, beta, E);
    const u64 *tab = modup_table(c, lp);
    // own rows: copies of the evaluation-form input
    if (!own_done) {
        dim3 grid((N + 255) / 256, lp, B);
        prof_begin(c);
        modup_own_kernel<<<grid, 256, 0, c->stream>>>(D, xe, xe_bstride, lp, c->K, c->alpha, beta, c->logn);
        note_launch(c, "modup", 16.0 * N * (double)B * lp);
    }
    // every other row: base conversion of its digit fused with the forward NTT
    std::string key = fmt("modup_rows:%u:%u", B, lp);
    std::vector<u32> rows;
    for (u32 b = 0; b < B; ++b)
        for (u32 j = 0; j < beta; ++j) {
            u32 lo = j * c->alpha, hi = std::min(lo + c->alpha, lp);
            for (u32 t = 0; t < E; ++t) {
                if (t >= lo && t < hi) continue;
                u32 prime = t < lp ? t : c->L1 + (t - lp);
                rows.push_back(((((u32)b * beta + j) * E + t) << 8) | prime);
            }
        }
    RowSet rs = rows_list(c, key, rows);
    if (rs.n == 0) return;
    // the digit rows read (mostly from L2), each converted row written once; butterflies of its NTT
    const double bytes = 8.0 * N * (double)rs.n * (1.0 + c->alpha), bfly = (double)rs.n * (N / 2);
    const int sp = ntt_layout(c, TUNE_NTT);
    if (sp == NTT_TWO_KERNEL) {
        prof_begin(c);
        NTT2_OUTER_LAUNCH(c, modup2_outer_kernel, c->logn, rs.n, D, (const u64 *)xc.p, rs, lp, c->K, c->alpha, beta,
                          tab, (const u64 *)c->tw, (const PrimeDev *)c->pdev);
        note_launch(c, "modup_ntt", bytes * c->alpha / (1.0 + c->alpha), bfly * (c->logn - NTT2_INNER_LOGN));
        prof_begin(c);
        ntt2_inner(c, D, rs, 0);
        note_launch(c, "modup_ntt", bytes / (1.0 + c->alpha), bfly * NTT2_INNER_LOGN);
        return;
    }
    prof_begin(c);
    launch_parts(c, modup_ntt_kernel<0>, modup_ntt_kernel<1>, dim3(rs.n), sp, ntt_part_threads(c->logn, sp),
                 ntt_part_smem(c->logn, sp), D, (const u64 *)xc.p, rs, lp, c->K, c->alpha, beta, c->logn, tab,
                 (const u64 *)c->tw, (const PrimeDev *)c->pdev);
    note_launch(c, "modup_ntt", bytes, bfly * c->logn);
}

static const u64 *pmod_table(Ctx *c);

// acc [S][B][2][lp+K][N] = sum_j sigma_{g_s}(D_j) (o) key_s,j (+ P * (padd0, padd1) when padd is given)
void ks_inner(Ctx *c, u64 *acc, const u64 *D, const KeyList &kl, u32 S, u32 B, u32 lp, const u64 *padd,
              size_t padd_bstride) {
    const u32 N = c->N, E = lp + c->K;
    dim3 grid((N + 255) / 256, E, S * B);
    prof_begin(c);
    ks_inner_kernel<<<grid, 256, 0, c->stream>>>(acc, D, kl, B, ks_digits(c, lp), lp, c->K, c->L1, c->logn, c->pdev,
                                                 padd, padd_bstride, padd ? pmod_table(c) : nullptr);
    {
        const double beta = ks_digits(c, lp);
        // digits read once, each step's key read once, accumulators written once (+ the addends read once)
        note_launch(c, "ks_inner", 8.0 * N * ((double)B * beta * E + (double)S * 2 * beta * E + (double)S * B * 2 * E +
                                              (padd ? (double)S * B * 2 * lp : 0.0)));
    }
}

// [P]_{q_t} with Shoup companions for the data primes
static const u64 *pmod_table(Ctx *c) {
    std::string key = "Pq";
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second.p;
    std::vector<u64> h(2 * c->L1);
    for (u32 t = 0; t < c->L1; ++t) {
        u64 q = c->primes[t], v = 1;
        for (u32 k = 0; k < c->K; ++k) v = mulmod_h(v, c->primes[c->L1 + k] % q, q);
        h[2 * t] = v;
        h[2 * t + 1] = shoup_h(v, q);
    }
    return c->const_table(key, h);
}

// [P 2^64]_{q_t} with Shoup companions for the data primes (P in Montgomery form)
static const u64 *pmont_table(Ctx *c) {
    std::string key = "PqMont";
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second.p;
    std::vector<u64> h(2 * c->L1);
    for (u32 t = 0; t < c->L1; ++t) {
        u64 q = c->primes[t], v = 1;
        for (u32 k = 0; k < c->K; ++k) v = mulmod_h(v, c->primes[c->L1 + k] % q, q);
        h[2 * t] = (u64)(((unsigned __int128)v << 64) % q);
        h[2 * t + 1] = shoup_h(h[2 * t], q);
    }
    return c->const_table(key, h);
}

// acc [S][B][2][lp+K][N]: lazy key-switch accumulators of the steps in kl (key nullptr, g = 1: identity)
void ks_lazy(Ctx *c, u64 *acc, const u64 *D, const u64 *x, const KeyList &kl, u32 S, u32 B, u32 lp) {
    const u32 N = c->N, E = lp + c->K;
    const u32 beta = ks_digits(c, lp);
    const int bt = tune_get(c, TUNE_LAZY_BT, 2), order = tune_get(c, TUNE_LAZY_ORDER, 0);
    const int maxd = beta <= 2 ? 2 : beta <= 4 ? 4 : 8;
    bool perm = beta <= 8 && (B + bt - 1) / bt <= 65535;
    for (u32 s = 0; s < S; ++s) {
        if (kl.g[s] != 1 && !kl.keyp[s]) perm = false;
        if (kl.g[s] != 1 && !D) throw HeError(HE_EINVAL, "ks_lazy: a key-switched step without ModUp digits");
    }
    prof_begin(c);
    if (perm) {
        const u32 nt = (N + 255) / 256, nb = (B + bt - 1) / bt;
        dim3 grid(order ? nb : nt, order ? nt : nb, E);
#define LAZY_LAUNCH(BTV, MD)                                                                                   \
    ks_lazy_perm_kernel<BTV, MD><<<grid, 256, (size_t)2 * 2 * MD * 256 * 8, c->stream>>>(                     \
        acc, D, x, kl, S, B, beta, lp, c->K, c->L1, c->logn, order, pmod_table(c), c->pdev)
        if (maxd == 8) {
            if (bt == 1) LAZY_LAUNCH(1, 8); else if (bt == 2) LAZY_LAUNCH(2, 8); else LAZY_LAUNCH(4, 8);
        } else if (maxd == 4) {
            if (bt == 1) LAZY_LAUNCH(1, 4); else if (bt == 2) LAZY_LAUNCH(2, 4); else LAZY_LAUNCH(4, 4);
        } else {
            if (bt == 1) LAZY_LAUNCH(1, 2); else if (bt == 2) LAZY_LAUNCH(2, 2); else LAZY_LAUNCH(4, 2);
        }
#undef LAZY_LAUNCH
    } else {
        dim3 grid((N + 255) / 256, E, S * B);
        ks_lazy_kernel<<<grid, 256, 0, c->stream>>>(acc, D, x, kl, B, beta, lp, c->K, c->L1, c->logn, pmod_table(c),
                                                     c->pdev);
    }
    note_launch(c, "ks_lazy",
                8.0 * N * ((double)B * beta * E + (double)S * 2 * beta * E + (double)B * 2 * lp + (double)S * B * 2 * E),
                (double)S * B * E * N * 2 * beta);
}

// the division of acc [S][B][2][lp+K][N] by the dropped basis (KD rows from dbase) onto lpo output
// limbs, in the tuned limb layout; bytes = the algorithmic bytes of the operation
static void moddown_launch(Ctx *c, u64 *out, u64 *acc, const u64 *addend, size_t addend_bstride, u32 add_mask,
                           const KeyList &kl, u32 S, u32 B, u32 lp, u32 dbase, u32 KD, u32 lpo, const u64 *tab,
                           double bytes) {
    const u32 N = c->N;
    const double bfly = (double)S * B * 2 * lpo * (N / 2);
    const int sp = ntt_layout(c, TUNE_MODDOWN);
    if (sp == NTT_TWO_KERNEL) {
        const u32 rows = S * B * 2 * lpo;
        prof_begin(c);
        NTT2_OUTER_LAUNCH(c, moddown2_outer_kernel, c->logn, rows, out, (const u64 *)acc, lp, c->K, c->L1, dbase,
                          KD, lpo, tab, (const u64 *)c->tw, (const PrimeDev *)c->pdev);
        note_launch(c, "moddown", bytes / 2, bfly * (c->logn - NTT2_INNER_LOGN));
        prof_begin(c);
        moddown2_inner_kernel<<<dim3(rows, N >> NTT2_INNER_LOGN), NTT2_INNER_THREADS, 0, c->stream>>>(
            out, (const u64 *)acc, addend, addend_bstride, add_mask, kl, B, lp, c->K, c->L1, KD, lpo, c->logn, tab,
            (const u64 *)c->tw, (const PrimeDev *)c->pdev);
        note_launch(c, "moddown", bytes / 2, bfly * NTT2_INNER_LOGN);
        return;
    }
    dim3 grid(lpo, 2, S * B);
    prof_begin(c);
    launch_parts(c, moddown_kernel<0>, moddown_kernel<1>, grid, sp, ntt_part_threads(c->logn, sp),
                 ntt_part_smem(c->logn, sp), out, (const u64 *)acc, addend, addend_bstride, add_mask, kl, B, lp,
                 c->K, c->L1, dbase, KD, lpo, c->logn, tab, (const u64 *)c->tw, (const PrimeDev *)c->pdev);
    note_launch(c, "moddown", bytes, bfly * c->logn);
}

// Z = the hoisted combination of the steps of kl (at most KEYLIST_MAX), accumulated in one pass;
// w null: one plain sum per input ciphertext (ks_comb_lazy_kernel), else one weighted output
// summed over the CH channels, w [S*CH][E][N] (O must be 1; w_ostride is not used): with one
// channel and enough ciphertexts the weights are folded into the keys (ks_fold_kernel, then
// ks_comb_lazy_kernel), otherwise ks_comb_kernel
void ks_comb(Ctx *c, u64 *Z, const u64 *D, const u64 *x, const KeyList &kl, u32 S, u32 CH, u32 B, u32 lp,
             const u64 *w, u32 O, size_t w_ostride, int accumulate) {
    const u32 N = c->N, E = lp + c->K, beta = ks_digits(c, lp);
    const bool weighted = w != nullptr;
    if (weighted && O != 1) throw HeError(HE_EINVAL, "ks_comb: one weighted output");
    if (S > KEYLIST_MAX) throw HeError(HE_EINVAL, "ks_comb: too many steps in one launch");
    u32 nks = 0;
    for (u32 s = 0; s < S; ++s)
        if (kl.g[s] != 1) {
            if (!kl.key[s] || !D) throw HeError(HE_EINVAL, "ks_comb: a key-switched step without key or digits");
            ++nks;
        }
    // ciphertexts per thread (tuned): 4 shares every key word between more products, 2 keeps
    // three CTAs per SM
    const u32 bt = tune_get(c, TUNE_COMB_BT, 4) == 2 ? 2 : 4;
    const u32 nb = weighted ? B : CH * B;
    const dim3 grid((N + 255) / 256, (nb + bt - 1) / bt, E);
    if (grid.y > 65535) throw HeError(HE_EINVAL, "ks_comb: batch too large for one launch");
    // digits unrolled up to 8 (the key words of a step held in registers), any count otherwise
    const int md = beta <= 4 ? 4 : beta <= 8 ? 8 : 0;
    const double Bt = (double)CH * B;
    // The lazy form (one reduction per output): plain sums, and weighted sums of one channel over
    // enough ciphertexts to pay for folding the weights into the keys (S*2*beta*E*N products,
    // against nb times that in the combination)
    const int fold_min = tune_get(c, TUNE_COMB_FOLD, COMB_FOLD_MIN_B);
    const bool fold = weighted && CH == 1 && (int)B >= std::max(1, fold_min);
    if (!weighted || fold) {
        // one step adds at most beta + 1 products to a 128-bit sum, folded before 63 could overflow it
        if (beta + 1 > 63) throw HeError(HE_EINVAL, "ks_comb: too many digits for one 128-bit sum");
        DBuf F, PW;
        KeyList kf = kl;
        u32 krow_sp = c->L1;
        size_t kst = (size_t)(c->L1 + c->K) * N;
        const u64 *pw = nullptr;
        if (fold) {
            if (nks) F = DBuf(c, (size_t)S * beta * 2 * E * N);
            PW = DBuf(c, (size_t)S * lp * N);
            prof_begin(c);
            ks_fold_kernel<<<dim3((N + 255) / 256, E, S), 256, 0, c->stream>>>(
                F.p, PW.p, kl, w, beta, lp, c->K, c->L1, c->logn, pmont_table(c), c->pdev);
            // the keys read and their folded copies written, the weights read, pw written
            note_launch(c, "ks_fold", 8.0 * N * (nks * 4.0 * beta * E + (double)S * E + (double)S * lp));
            for (u32 s = 0; s < S; ++s)
                if (kl.g[s] != 1) kf.key[s] = F.p + (size_t)s * beta * 2 * E * N;
            krow_sp = lp;
            kst = (size_t)E * N;
            pw = PW.p;
        }
        prof_begin(c);
#define LAZY_LAUNCH(BTV, MDV)                                                                                    \
    ks_comb_lazy_kernel<BTV, MDV><<<grid, 256, 0, c->stream>>>(Z, D, x, kf, S, nb, beta, lp, c->K, c->L1, krow_sp, \
                                                              kst, pw, pmont_table(c), accumulate, c->logn,     \
                                                              c->pdev)
        if (bt == 2) {
            if (md == 4) LAZY_LAUNCH(2, 4); else if (md == 8) LAZY_LAUNCH(2, 8); else LAZY_LAUNCH(2, 0);
        } else {
            if (md == 4) LAZY_LAUNCH(4, 4); else if (md == 8) LAZY_LAUNCH(4, 8); else LAZY_LAUNCH(4, 0);
        }
#undef LAZY_LAUNCH
        // the digits, keys (or folded keys and pw) and the inputs read once, the outputs written
        // once; 64x64->128 multiply-accumulates: the key products and one c0 product per step
        note_launch(c, "ks_comb",
                    8.0 * N * (Bt * beta * E + nks * 2.0 * beta * E + (fold ? (double)S * lp : 0) + Bt * lp +
                               Bt * 2 * E * (accumulate ? 2 : 1)),
                    (double)N * (2.0 * E * nks * Bt * beta + Bt * S * lp));
        return;
    }
    prof_begin(c);
#define COMB_LAUNCH(BTV, MDV)                                                                                   \
    ks_comb_kernel<BTV, MDV><<<grid, 256, 0, c->stream>>>(Z, D, x, kl, S, CH, B, beta, lp, c->K, c->L1, c->logn,  \
                                                          w, accumulate, pmod_table(c), c->pdev)
    if (bt == 2) {
        if (md == 4) COMB_LAUNCH(2, 4); else if (md == 8) COMB_LAUNCH(2, 8); else COMB_LAUNCH(2, 0);
    } else {
        if (md == 4) COMB_LAUNCH(4, 4); else if (md == 8) COMB_LAUNCH(4, 8); else COMB_LAUNCH(4, 0);
    }
#undef COMB_LAUNCH
    // the digits, keys, weights and the inputs' c0 read once, the outputs written once; 64x64->128
    // multiply-accumulates of the key products and of the weights
    note_launch(c, "ks_comb",
                8.0 * N * (Bt * beta * E + nks * 2.0 * beta * E + (double)O * S * CH * E + Bt * lp +
                           (double)O * 2 * E * (accumulate ? 2 : 1)),
                (double)N * E * 2 * (nks * Bt * beta + (double)O * S * CH * B));
}

// out [S][B][2][lp][N] = ModDown(acc) (+ addend: poly k of ct b gathered by sigma_{g_s} when add_mask bit k)
void ks_moddown(Ctx *c, u64 *out, u64 *acc, const u64 *addend, size_t addend_bstride, u32 add_mask,
                const KeyList &kl, u32 S, u32 B, u32 lp) {
    const u32 N = c->N, E = lp + c->K;
    // inverse NTT of the special-prime rows of acc
    std::string key = fmt("md_rows:%u:%u:%u", S, B, lp);
    std::vector<u32> rows;
    for (u32 sb = 0; sb < S * B; ++sb)
        for (u32 k = 0; k < 2; ++k)
            for (u32 kk = 0; kk < c->K; ++kk) rows.push_back((((sb * 2 + k) * E + lp + kk) << 8) | (c->L1 + kk));
    ntt_inverse(c, acc, rows_list(c, key, rows));
    moddown_launch(c, out, acc, addend, addend_bstride, add_mask, kl, S, B, lp, lp, c->K, lp, moddown_table(c),
                   8.0 * N * (double)S * B * (2.0 * E + (addend ? __builtin_popcount(add_mask) : 0) * lp + 2.0 * lp));
}

// out [nct][2][lp-1][N] = ModDown and rescale of acc [nct][2][lp+K][N] as one division by q_top * P
void ks_moddown_rescale(Ctx *c, u64 *out, u64 *acc, u32 nct, u32 lp) {
    const u32 N = c->N, E = lp + c->K;
    if (lp < 2) throw HeError(HE_ELEVEL, "rescale: no level left");
    // inverse NTT of the dropped rows: the top data limb and the special limbs
    std::string key = fmt("mdrs_rows:%u:%u", nct, lp);
    std::vector<u32> rows;
    for (u32 b = 0; b < nct; ++b)
        for (u32 k = 0; k < 2; ++k) {
            rows.push_back((((b * 2 + k) * E + lp - 1) << 8) | (lp - 1));
            for (u32 kk = 0; kk < c->K; ++kk) rows.push_back((((b * 2 + k) * E + lp + kk) << 8) | (c->L1 + kk));
        }
    ntt_inverse(c, acc, rows_list(c, key, rows));
    KeyList none;
    none.g[0] = 1;
    none.key[0] = nullptr;
    moddown_launch(c, out, acc, nullptr, 0, 0, none, 1, nct, lp, lp - 1, c->K + 1, lp - 1,
                   moddown_rescale_table(c, lp), 8.0 * N * (double)nct * (2.0 * E + 2.0 * (lp - 1)));
}

// out [B][2][lp-1][N] = rescale(in [B][2][lp][N])
void rescale_batch(Ctx *c, u64 *out, const u64 *in, u32 B, u32 lp) {
    const u32 N = c->N;
    if (lp < 2) throw HeError(HE_ELEVEL, "rescale: no level left");
    DBuf top(c, (size_t)B * 2 * N);
    gather_rows(c, top.p, in + (size_t)(lp - 1) * N, B * 2, lp);
    ntt_inverse(c, top.p, rows_regular(B * 2, 1, 0, lp - 1));
    const double bytes = 8.0 * N * (double)B * 2 * (lp + 1 + lp - 1), bfly = (double)B * 2 * (lp - 1) * (N / 2);
    const int sp = ntt_layout(c, TUNE_RESCALE);
    if (sp == NTT_TWO_KERNEL) {
        const u32 rows = B * 2 * (lp - 1);
        prof_begin(c);
        NTT2_OUTER_LAUNCH(c, rescale2_outer_kernel, c->logn, rows, out, (const u64 *)top.p, lp, (const u64 *)c->tw,
                          (const PrimeDev *)c->pdev);
        note_launch(c, "rescale", bytes / 2, bfly * (c->logn - NTT2_INNER_LOGN));
        prof_begin(c);
        rescale2_inner_kernel<<<dim3(rows, N >> NTT2_INNER_LOGN), NTT2_INNER_THREADS, 0, c->stream>>>(
            out, in, lp, c->logn, rescale_table(c, lp), (const u64 *)c->tw, (const PrimeDev *)c->pdev);
        note_launch(c, "rescale", bytes / 2, bfly * NTT2_INNER_LOGN);
        return;
    }
    dim3 grid(lp - 1, 2, B);
    prof_begin(c);
    launch_parts(c, rescale_kernel<0>, rescale_kernel<1>, grid, sp, ntt_part_threads(c->logn, sp), ntt_part_smem(c->logn, sp), out, in,
                 (const u64 *)top.p, lp, c->logn, rescale_table(c, lp), (const u64 *)c->tw, (const PrimeDev *)c->pdev);
    note_launch(c, "rescale", bytes, bfly * c->logn);
}
