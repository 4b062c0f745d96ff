/*
 * ckks_ref.c -- plain, slow CPU oracle for the RNS-CKKS ring arithmetic that
 * UniHENN's encrypted CNN layers run on (paper Sec. II-B: Add/Mul/Rot on CKKS
 * ciphertexts; the RNS/hybrid-key-switching details follow Cheon-Han-Kim-Kim-Song
 * 2018 and Han-Ki 2020, which the paper relies on through SEAL).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this file.  It shares no code, header or
 * table with the CUDA library and never calls it.
 *
 * Style: every modular product is `(unsigned __int128)a * b % q`; every routine
 * is the textbook definition written out (no lazy reduction, no Shoup/Barrett,
 * no blocking).  Limbs are arrays of n uint64 residues in [0, q).
 * Evaluation ("NTT") form is NATURAL order: slot k holds a(psi^(2k+1)).
 * The FP64 encoder follows the canonical embedding (paper Sec. II-B, CKKS) and
 * must be compiled with -ffp-contract=off so every double op rounds once.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ scalar */

u64 o_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : (u64)((u128)a + q - b); }

u64 o_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = o_mulmod(r, a, q);
        a = o_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* q prime: Fermat inverse */
u64 o_invmod(u64 a, u64 q) { return o_powmod(a, q - 2, q); }

/* signed integer -> residue in [0, q) */
static u64 red_signed(i64 v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) + 1; /* |v| without overflow */
    m %= q;
    return m ? q - m : 0;
}

/* ------------------------------------------------------------------ NTT */
/* Forward negacyclic transform, written as "twist by psi^j, then a cyclic
 * length-n DFT with omega = psi^2" (radix-2 decimation in time on the
 * bit-reversed input):  out[k] = sum_j a[j] * psi^(j*(2k+1)) mod q.          */
static void bitrev_permute(u64 *a, int logn) {
    int n = 1 << logn;
    for (int i = 0; i < n; i++) {
        int r = 0;
        for (int b = 0; b < logn; b++) r |= ((i >> b) & 1) << (logn - 1 - b);
        if (r > i) { u64 t = a[i]; a[i] = a[r]; a[r] = t; }
    }
}

static void cyclic_dft(u64 *a, int logn, u64 q, u64 omega) {
    int n = 1 << logn;
    bitrev_permute(a, logn);
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = o_powmod(omega, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 w = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = o_mulmod(a[i + j + len / 2], w, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                w = o_mulmod(w, wl, q);
            }
        }
    }
}

void o_ntt(u64 *a, int logn, u64 q, u64 psi) {
    int n = 1 << logn;
    u64 pw = 1;
    for (int j = 0; j < n; j++) { a[j] = o_mulmod(a[j], pw, q); pw = o_mulmod(pw, psi, q); }
    cyclic_dft(a, logn, q, o_mulmod(psi, psi, q));
}

/* inverse: cyclic inverse DFT (omega^-1), times n^-1, untwist by psi^-j */
void o_intt(u64 *a, int logn, u64 q, u64 psi) {
    int n = 1 << logn;
    u64 psi_inv = o_invmod(psi, q);
    cyclic_dft(a, logn, q, o_mulmod(psi_inv, psi_inv, q));
    u64 ninv = o_invmod((u64)n % q, q);
    u64 pw = ninv;
    for (int j = 0; j < n; j++) { a[j] = o_mulmod(a[j], pw, q); pw = o_mulmod(pw, psi_inv, q); }
}

/* batched helpers: limb l of a[nl][n] uses q[l], psi[l] */
void o_ntt_limbs(u64 *a, int nl, int logn, const u64 *q, const u64 *psi) {
    for (int l = 0; l < nl; l++) o_ntt(a + ((size_t)l << logn), logn, q[l], psi[l]);
}
void o_intt_limbs(u64 *a, int nl, int logn, const u64 *q, const u64 *psi) {
    for (int l = 0; l < nl; l++) o_intt(a + ((size_t)l << logn), logn, q[l], psi[l]);
}

/* ------------------------------------------------------------- pointwise */
void o_mul(u64 *out, const u64 *a, const u64 *b, int nl, int n, const u64 *q) {
    for (int l = 0; l < nl; l++)
        for (int i = 0; i < n; i++) {
            size_t k = (size_t)l * n + i;
            out[k] = o_mulmod(a[k], b[k], q[l]);
        }
}
void o_add(u64 *out, const u64 *a, const u64 *b, int nl, int n, const u64 *q) {
    for (int l = 0; l < nl; l++)
        for (int i = 0; i < n; i++) {
            size_t k = (size_t)l * n + i;
            out[k] = addmod(a[k], b[k], q[l]);
        }
}
void o_sub(u64 *out, const u64 *a, const u64 *b, int nl, int n, const u64 *q) {
    for (int l = 0; l < nl; l++)
        for (int i = 0; i < n; i++) {
            size_t k = (size_t)l * n + i;
            out[k] = submod(a[k], b[k], q[l]);
        }
}
/* out += a*b (the multiply-accumulate of a plaintext mask into a sum) */
void o_muladd(u64 *acc, const u64 *a, const u64 *b, int nl, int n, const u64 *q) {
    for (int l = 0; l < nl; l++)
        for (int i = 0; i < n; i++) {
            size_t k = (size_t)l * n + i;
            acc[k] = addmod(acc[k], o_mulmod(a[k], b[k], q[l]), q[l]);
        }
}
/* signed small integers (ternary / error / encoded message) into residues */
void o_reduce_signed(u64 *out, const i64 *v, int nl, int n, const u64 *q) {
    for (int l = 0; l < nl; l++)
        for (int i = 0; i < n; i++) out[(size_t)l * n + i] = red_signed(v[i], q[l]);
}

/* --------------------------------------------------------- automorphisms */
/* X -> X^g on the coefficient form: coefficient j moves to j*g mod 2n,
 * with a sign flip when that exponent lands in [n, 2n) (X^n = -1).        */
void o_automorph_coeff(u64 *out, const u64 *in, int nl, int logn, u64 g, const u64 *q) {
    int n = 1 << logn;
    u64 twon = 2 * (u64)n;
    for (int l = 0; l < nl; l++) {
        const u64 *a = in + (size_t)l * n;
        u64 *o = out + (size_t)l * n;
        for (int j = 0; j < n; j++) {
            u64 e = ((u64)j * g) % twon;
            if (e < (u64)n) o[e] = a[j];
            else o[e - n] = a[j] ? q[l] - a[j] : 0;
        }
    }
}
/* same automorphism on natural-order evaluation form: slot k is a(psi^(2k+1));
 * sigma_g(a) at psi^(2k+1) equals a at psi^(g(2k+1)), i.e. slot (g(2k+1)-1)/2. */
void o_automorph_eval(u64 *out, const u64 *in, int nl, int logn, u64 g) {
    int n = 1 << logn;
    u64 twon = 2 * (u64)n;
    for (int l = 0; l < nl; l++)
        for (int k = 0; k < n; k++) {
            u64 e = (g * (2 * (u64)k + 1)) % twon;
            out[(size_t)l * n + k] = in[(size_t)l * n + (e - 1) / 2];
        }
}

/* ----------------------------------------------------- base conversion */
/* Fast base conversion (Bajard et al. 2016 / Halevi-Polyakov-Shoup 2018),
 * no correction term: for input residues x_i modulo qin_i (coefficient form)
 *   y_t = sum_i [x_i * qhat_i^{-1}]_{qin_i} * qhat_i  mod qout_t,
 * with qhat_i = prod_{k != i} qin_k.                                         */
void o_bconv(u64 *out, const u64 *in, int nin, const u64 *qin, int nout, const u64 *qout, int n) {
    u64 *hinv = (u64 *)malloc(sizeof(u64) * nin);
    u64 *hmod = (u64 *)malloc(sizeof(u64) * nin * (nout ? nout : 1));
    for (int i = 0; i < nin; i++) {
        u64 h = 1;
        for (int k = 0; k < nin; k++) if (k != i) h = o_mulmod(h, qin[k] % qin[i], qin[i]);
        hinv[i] = o_invmod(h, qin[i]);
        for (int t = 0; t < nout; t++) {
            u64 m = 1;
            for (int k = 0; k < nin; k++) if (k != i) m = o_mulmod(m, qin[k] % qout[t], qout[t]);
            hmod[i * nout + t] = m;
        }
    }
    for (int t = 0; t < nout; t++)
        for (int c = 0; c < n; c++) {
            u64 acc = 0;
            for (int i = 0; i < nin; i++) {
                u64 v = o_mulmod(in[(size_t)i * n + c], hinv[i], qin[i]);
                acc = addmod(acc, o_mulmod(v % qout[t], hmod[i * nout + t], qout[t]), qout[t]);
            }
            out[(size_t)t * n + c] = acc;
        }
    free(hinv);
    free(hmod);
}

/* ------------------------------------------------------------ rescale */
/* Divide by the top prime q_top with the centred remainder (RNS rescale of
 * CKKS): r = [c_top]_{q_top} lifted to (-q_top/2, q_top/2]; for each lower
 * limb c'_i = (c_i - r) * q_top^{-1} mod q_i.   in: nl limbs eval form,
 * out: nl-1 limbs eval form.  psi[] are the limbs' roots.                    */
void o_rescale(u64 *out, const u64 *in, int nl, int logn, const u64 *q, const u64 *psi) {
    int n = 1 << logn;
    u64 qt = q[nl - 1];
    u64 *top = (u64 *)malloc(sizeof(u64) * n);
    u64 *r = (u64 *)malloc(sizeof(u64) * n);
    memcpy(top, in + (size_t)(nl - 1) * n, sizeof(u64) * n);
    o_intt(top, logn, qt, psi[nl - 1]);
    for (int i = 0; i < nl - 1; i++) {
        for (int c = 0; c < n; c++) {
            i64 v = top[c] > qt / 2 ? (i64)top[c] - (i64)qt : (i64)top[c];
            r[c] = red_signed(v, q[i]);
        }
        o_ntt(r, logn, q[i], psi[i]);
        u64 qinv = o_invmod(qt % q[i], q[i]);
        for (int c = 0; c < n; c++)
            out[(size_t)i * n + c] = o_mulmod(submod(in[(size_t)i * n + c], r[c], q[i]), qinv, q[i]);
    }
    free(top);
    free(r);
}

/* ------------------------------------------------------------ ModDown */
/* acc: (nq + np) limbs eval form over q_0..q_{nq-1}, p_0..p_{np-1}.
 * out_i = (acc_i - BConv_{P->q_i}([acc]_P)) * P^{-1} mod q_i (eval form). */
void o_moddown(u64 *out, const u64 *acc, int nq, int np, int logn,
               const u64 *q, const u64 *qpsi, const u64 *p, const u64 *ppsi) {
    int n = 1 << logn;
    u64 *pc = (u64 *)malloc(sizeof(u64) * (size_t)np * n);
    u64 *cv = (u64 *)malloc(sizeof(u64) * (size_t)nq * n);
    memcpy(pc, acc + (size_t)nq * n, sizeof(u64) * (size_t)np * n);
    o_intt_limbs(pc, np, logn, p, ppsi);
    o_bconv(cv, pc, np, p, nq, q, n);
    o_ntt_limbs(cv, nq, logn, q, qpsi);
    for (int i = 0; i < nq; i++) {
        u64 pm = 1;
        for (int k = 0; k < np; k++) pm = o_mulmod(pm, p[k] % q[i], q[i]);
        u64 pinv = o_invmod(pm, q[i]);
        for (int c = 0; c < n; c++)
            out[(size_t)i * n + c] =
                o_mulmod(submod(acc[(size_t)i * n + c], cv[(size_t)i * n + c], q[i]), pinv, q[i]);
    }
    free(pc);
    free(cv);
}

/* --------------------------------------------------------------- ModUp */
/* One digit of hybrid key switching: x (eval form) limbs [lo, hi) of the
 * active chain q_0..q_{nq-1}; output (nq + np) limbs eval form over
 * q_0..q_{nq-1}, p_0..p_{np-1}: the digit's own limbs are copied, every other
 * limb is the fast base conversion of the digit (coefficient form) followed
 * by the forward transform.                                                   */
void o_modup_digit(u64 *out, const u64 *x, int lo, int hi, int nq, int np, int logn,
                   const u64 *q, const u64 *qpsi, const u64 *p, const u64 *ppsi) {
    int n = 1 << logn;
    int nd = hi - lo, nt = nq - nd + np;
    u64 *dc = (u64 *)malloc(sizeof(u64) * (size_t)nd * n);
    u64 *tq = (u64 *)malloc(sizeof(u64) * (nt ? nt : 1));
    u64 *tpsi = (u64 *)malloc(sizeof(u64) * (nt ? nt : 1));
    u64 *y = (u64 *)malloc(sizeof(u64) * (size_t)(nt ? nt : 1) * n);
    memcpy(dc, x + (size_t)lo * n, sizeof(u64) * (size_t)nd * n);
    o_intt_limbs(dc, nd, logn, q + lo, qpsi + lo);
    int t = 0;
    for (int i = 0; i < nq; i++) if (i < lo || i >= hi) { tq[t] = q[i]; tpsi[t] = qpsi[i]; t++; }
    for (int k = 0; k < np; k++) { tq[t] = p[k]; tpsi[t] = ppsi[k]; t++; }
    o_bconv(y, dc, nd, q + lo, nt, tq, n);
    o_ntt_limbs(y, nt, logn, tq, tpsi);
    t = 0;
    for (int i = 0; i < nq + np; i++) {
        u64 *dst = out + (size_t)i * n;
        if (i >= lo && i < hi) memcpy(dst, x + (size_t)i * n, sizeof(u64) * n);
        else { memcpy(dst, y + (size_t)t * n, sizeof(u64) * n); t++; }
    }
    free(dc); free(tq); free(tpsi); free(y);
}

/* ----------------------------------------------------------- sampling */
/* Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014, with the
 * "variant 13" finaliser): the stream state is output #stream of a
 * SplitMix64 seeded with `seed`; word i is output #i of a SplitMix64 seeded
 * with that state.                                                           */
#define SM_GAMMA 0x9e3779b97f4a7c15ULL
static u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
u64 o_rand_word(u64 seed, u64 stream, u64 i) {
    u64 s = sm_mix(seed + (stream + 1) * SM_GAMMA);
    return sm_mix(s + (i + 1) * SM_GAMMA);
}
/* ternary {-1,0,1}: (r mod 3) - 1 */
void o_sample_ternary(i64 *out, u64 seed, u64 stream, int n) {
    for (int i = 0; i < n; i++) out[i] = (i64)(o_rand_word(seed, stream, (u64)i) % 3) - 1;
}
/* centred binomial, eta = 21: popcount of 21 bits minus popcount of the next 21 */
void o_sample_cbd(i64 *out, u64 seed, u64 stream, int n) {
    for (int i = 0; i < n; i++) {
        u64 r = o_rand_word(seed, stream, (u64)i);
        out[i] = (i64)__builtin_popcountll(r & 0x1FFFFFULL) - (i64)__builtin_popcountll((r >> 21) & 0x1FFFFFULL);
    }
}
/* uniform mod q: floor(r * q / 2^64) */
void o_sample_uniform(u64 *out, u64 seed, u64 stream, int n, u64 q) {
    for (int i = 0; i < n; i++) out[i] = (u64)(((u128)o_rand_word(seed, stream, (u64)i) * q) >> 64);
}

/* ------------------------------------------------------ FP64 encoder */
/* Canonical-embedding encoder for N = 2M (CKKS, paper Sec. II-B).  Slot j is
 * the value at zeta^(5^j), zeta = exp(i*pi/N).  Writing c_k = m_k + i*m_{k+M}
 * (k < M), every slot point t = 5^j mod 2N is 1 mod 4, and
 *     m(zeta^t) = sum_k (c_k zeta^k) w^(s k),  w = exp(2*pi*i/M), s = (t-1)/4,
 * i.e. a length-M DFT of the twisted vector.  Encoding inverts it:
 * place z_j at s_j, inverse DFT (unnormalised, radix-2 DIT on bit-reversed
 * input), untwist by conj(zeta^k), scale by Delta/M, round half to even.
 * Twiddles: cos/sin of (2*pi*k)/M and (pi*k)/N evaluated exactly as written.
 * Complex product (a+bi)(c+di) = (ac - bd) + (ad + bc)i, each op rounded.   */
static void fft_dit(double *re, double *im, int logm, int inverse) {
    int m = 1 << logm;
    double *wr_t = (double *)malloc(sizeof(double) * (m / 2 + 1));
    double *wi_t = (double *)malloc(sizeof(double) * (m / 2 + 1));
    for (int k = 0; k < m / 2; k++) {
        double ang = 2.0 * M_PI * (double)k / (double)m;
        wr_t[k] = cos(ang);
        wi_t[k] = inverse ? -sin(ang) : sin(ang);
    }
    for (int i = 0; i < m; i++) {
        int r = 0;
        for (int b = 0; b < logm; b++) r |= ((i >> b) & 1) << (logm - 1 - b);
        if (r > i) {
            double t = re[i]; re[i] = re[r]; re[r] = t;
            t = im[i]; im[i] = im[r]; im[r] = t;
        }
    }
    for (int h = 1; h < m; h <<= 1) {
        for (int b = 0; b < m; b += 2 * h) {
            for (int j = 0; j < h; j++) {
                int k = j * (m / (2 * h));
                double wr = wr_t[k], wi = wi_t[k];
                double ur = re[b + j], ui = im[b + j];
                double xr = re[b + j + h], xi = im[b + j + h];
                double vr = xr * wr - xi * wi;
                double vi = xr * wi + xi * wr;
                re[b + j] = ur + vr; im[b + j] = ui + vi;
                re[b + j + h] = ur - vr; im[b + j + h] = ui - vi;
            }
        }
    }
    free(wr_t);
    free(wi_t);
}

static int slot_pos(int j, int logn) {
    u64 twon = 2ULL << logn;
    u64 t = o_powmod(5, (u64)j, twon);
    return (int)((t - 1) / 4);
}

/* z (M complex values) -> rounded integer coefficients m[0..N).  Returns 0,
 * or -1 when a coefficient does not fit in a signed 64-bit integer.          */
int o_encode(i64 *m, const double *zre, const double *zim, int logn, double scale) {
    int N = 1 << logn, M = N / 2, logm = logn - 1;
    double *re = (double *)calloc(M, sizeof(double));
    double *im = (double *)calloc(M, sizeof(double));
    for (int j = 0; j < M; j++) {
        int s = slot_pos(j, logn);
        re[s] = zre[j];
        im[s] = zim ? zim[j] : 0.0;
    }
    fft_dit(re, im, logm, 1);
    double f = scale / (double)M;
    int rc = 0;
    for (int k = 0; k < M; k++) {
        double ang = M_PI * (double)k / (double)N;
        double tr = cos(ang), ti = -sin(ang);
        double cr = re[k] * tr - im[k] * ti;
        double ci = re[k] * ti + im[k] * tr;
        double a = nearbyint(cr * f), b = nearbyint(ci * f);
        if (!(fabs(a) < 9.2e18) || !(fabs(b) < 9.2e18)) rc = -1;
        m[k] = (i64)a;
        m[k + M] = (i64)b;
    }
    free(re);
    free(im);
    return rc;
}

/* coefficients (as doubles, already divided by the scale) -> M slot values */
void o_decode(double *zre, double *zim, const double *coef, int logn) {
    int N = 1 << logn, M = N / 2, logm = logn - 1;
    double *re = (double *)malloc(sizeof(double) * M);
    double *im = (double *)malloc(sizeof(double) * M);
    for (int k = 0; k < M; k++) {
        double ang = M_PI * (double)k / (double)N;
        double tr = cos(ang), ti = sin(ang);
        double ar = coef[k], ai = coef[k + M];
        re[k] = ar * tr - ai * ti;
        im[k] = ar * ti + ai * tr;
    }
    fft_dit(re, im, logm, 0);
    for (int j = 0; j < M; j++) {
        int s = slot_pos(j, logn);
        zre[j] = re[s];
        zim[j] = im[s];
    }
    free(re);
    free(im);
}
