// encode.cu -- CKKS canonical-embedding encoder / decoder in FP64 (paper
// Sec. II-B; Cheon et al. 2017), plus the packing of flattened samples
// (paper Sec. III-A/B) and the decryption combine.
//
// With M = N/2, c_k = m_k + i*m_{k+M} and zeta = exp(i*pi/N), every slot point
// zeta^(5^j) has exponent t = 1 mod 4, and m(zeta^t) = sum_k (c_k zeta^k) w^(s k)
// with w = exp(2*pi*i/M), s = (t-1)/4: a length-M DFT of the twisted vector.
// Encoding inverts it: place slot j at s_j, inverse DFT (radix-2 decimation in
// time on bit-reversed input), untwist by conj(zeta^k), multiply by Delta/M,
// round half to even.  Each butterfly and twist uses IEEE double operations
// in a fixed order (products first, one rounding per operation, no FMA), so
// the result is bit-reproducible.
#include "he_internal.cuh"
#include "ntt_block.cuh"
#include "ring.cuh"

// the FFT's share of one CTA: complex points [lo, lo + n) of M = N/2; split over
// a 2-CTA cluster exactly when the limb's NTT is (N = 2^15: 256 KiB of points)
template <int SPLIT>
__device__ __forceinline__ Part fft_part(int logn) {
    Part p;
    p.split = SPLIT;
    p.n = 1u << (logn - 1 - p.split);
    p.lo = SPLIT ? (blockIdx.x & 1u) * p.n : 0u;
    return p;
}

__device__ __forceinline__ void fft_bfly(double &ur, double &ui, double &xr, double &xi, double wr, double wi) {
    const double vr = __dsub_rn(__dmul_rn(xr, wr), __dmul_rn(xi, wi));
    const double vi = __dadd_rn(__dmul_rn(xr, wi), __dmul_rn(xi, wr));
    xr = __dsub_rn(ur, vr);
    xi = __dsub_rn(ui, vi);
    ur = __dadd_rn(ur, vr);
    ui = __dadd_rn(ui, vi);
}

// radix-2 decimation in time on bit-reversed input, length M = 2^logm; this CTA
// holds points [p.lo, p.lo + p.n).  Stages with half-span h < p.n are local; when
// the points are split over two CTAs the last stage (h = M/2) pairs local index j
// of CTA 0 with local index j of CTA 1 through distributed shared memory.
__device__ void part_fft(double *re, double *im, int logm, const double *__restrict__ w, bool inverse,
                         const Part &p) {
    const int nloc = logm - p.split;
    for (int lgh = 0; lgh < nloc; ++lgh) {
        const u32 h = 1u << lgh;
        for (u32 b = threadIdx.x; b < p.n / 2; b += blockDim.x) {
            const u32 j = b & (h - 1);
            const u32 base = (b >> lgh) << (lgh + 1);
            const u32 k = j << (logm - 1 - lgh);
            const double wr = w[2 * k];
            const double wi = inverse ? -w[2 * k + 1] : w[2 * k + 1];
            double ur = re[base + j], ui = im[base + j];
            double xr = re[base + j + h], xi = im[base + j + h];
            fft_bfly(ur, ui, xr, xi, wr, wi);
            re[base + j] = ur;
            im[base + j] = ui;
            re[base + j + h] = xr;
            im[base + j + h] = xi;
        }
        __syncthreads();
    }
    if (!p.split) return;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    double *re0 = cl.map_shared_rank(re, 0), *im0 = cl.map_shared_rank(im, 0);
    double *re1 = cl.map_shared_rank(re, 1), *im1 = cl.map_shared_rank(im, 1);
    const u32 j0 = p.lo / 2;
    for (u32 j = j0 + threadIdx.x; j < j0 + p.n / 2; j += blockDim.x) {
        const double wr = w[2 * j];
        const double wi = inverse ? -w[2 * j + 1] : w[2 * j + 1];
        double ur = re0[j], ui = im0[j], xr = re1[j], xi = im1[j];
        fft_bfly(ur, ui, xr, xi, wr, wi);
        re0[j] = ur;
        im0[j] = ui;
        re1[j] = xr;
        im1[j] = xi;
    }
    cl.sync();
}

__device__ __forceinline__ u64 red_signed(i64 v, const PrimeDev &P) {
    return v >= 0 ? reduce64((u64)v, P) : neg_mod(reduce64((u64)(-v), P), P.q);
}

// after the inverse FFT: untwist, scale, round, reduce into lp limbs
// (limb l < lpq: data prime l; limb l >= lpq: special prime pbase + l - lpq)
__device__ void encode_finish(const double *re, const double *im, u64 *out, u32 lp, int logn, double f,
                              const double *__restrict__ tw, const PrimeDev *__restrict__ pd, int *err,
                              const Part &pt, u32 lpq = 0xffffffffu, u32 pbase = 0) {
    const u32 N = 1u << logn, M = N / 2;
    for (u32 k = pt.lo + threadIdx.x; k < pt.lo + pt.n; k += blockDim.x) {
        const double tr = tw[2 * k], ti = -tw[2 * k + 1];
        const double xr = re[k - pt.lo], xi = im[k - pt.lo];
        const double cr = __dsub_rn(__dmul_rn(xr, tr), __dmul_rn(xi, ti));
        const double ci = __dadd_rn(__dmul_rn(xr, ti), __dmul_rn(xi, tr));
        const double a = __dmul_rn(cr, f), b = __dmul_rn(ci, f);
        if (!(fabs(a) < 9.2e18) || !(fabs(b) < 9.2e18)) {
            atomicExch(err, 1);
            continue;
        }
        const i64 ia = __double2ll_rn(a), ib = __double2ll_rn(b);
        for (u32 l = 0; l < lp; ++l) {
            const PrimeDev &P = pd[l < lpq ? l : pbase + (l - lpq)];
            out[(size_t)l * N + k] = red_signed(ia, P);
            out[(size_t)l * N + k + M] = red_signed(ib, P);
        }
    }
}

// dense slot vectors z[v][M] -> coefficient residues out[v][lp][N]
template <int SPLIT>
__global__ void __launch_bounds__(1024) encode_dense_kernel(u64 *out, const double *__restrict__ z, u32 lp,
                                                            int logn, double f, const double *__restrict__ fw,
                                                            const double *__restrict__ ft,
                                                            const u32 *__restrict__ pos_br,
                                                            const PrimeDev *__restrict__ pd, int *err) {
    extern __shared__ double smd[];
    const u32 N = 1u << logn, M = N / 2;
    const Part pt = fft_part<SPLIT>(logn);
    const u32 v = part_row<SPLIT>();
    double *re = smd, *im = smd + pt.n;
    const double *zv = z + (size_t)v * M;
    for (u32 j = threadIdx.x; j < M; j += blockDim.x) {
        const u32 p = pos_br[j] - pt.lo;
        if (p < pt.n) {
            re[p] = zv[j];
            im[p] = 0.0;
        }
    }
    __syncthreads();
    part_fft(re, im, logn - 1, fw, true, pt);
    encode_finish(re, im, out + (size_t)v * lp * N, lp, logn, f, ft, pd, err, pt);
}

// sparse slot vectors: vector v has entries [off[v], off[v+1]) of (pos, val),
// replicated at pos + s*stride for s < ns.
template <int SPLIT>
__global__ void __launch_bounds__(1024) encode_sparse_kernel(u64 *out, const u32 *__restrict__ off,
                                                             const u32 *__restrict__ pos,
                                                             const double *__restrict__ val, u32 stride, u32 ns,
                                                             u32 lp, int logn, double f, const double *__restrict__ fw,
                                                             const double *__restrict__ ft,
                                                             const u32 *__restrict__ pos_br,
                                                             const PrimeDev *__restrict__ pd, int *err, u32 lpq,
                                                             u32 pbase) {
    extern __shared__ double smd[];
    const u32 N = 1u << logn, M = N / 2;
    const Part pt = fft_part<SPLIT>(logn);
    const u32 v = part_row<SPLIT>();
    double *re = smd, *im = smd + pt.n;
    for (u32 j = threadIdx.x; j < pt.n; j += blockDim.x) {
        re[j] = 0.0;
        im[j] = 0.0;
    }
    __syncthreads();
    const u32 e0 = off[v], e1 = off[v + 1];
    const u32 cnt = (e1 - e0) * ns;
    for (u32 x = threadIdx.x; x < cnt; x += blockDim.x) {
        u32 e = e0 + x / ns, s = x % ns;
        u32 slot = pos[e] + s * stride;
        if (slot < M) {
            const u32 p = pos_br[slot] - pt.lo;
            if (p < pt.n) re[p] = val[e];
        }
    }
    __syncthreads();
    part_fft(re, im, logn - 1, fw, true, pt);
    encode_finish(re, im, out + (size_t)v * lp * N, lp, logn, f, ft, pd, err, pt, lpq, pbase);
}

// decode: coefficient-form limb q_0 of m (rows [v][N], residues) -> selected slots
// out[v][s][i] = slot (s*stride + i), i < nper, s < ns
template <int SPLIT>
__global__ void __launch_bounds__(1024) decode_kernel(double *out, const u64 *__restrict__ m, double scale,
                                                      u32 stride, u32 ns, u32 nper, int logn,
                                                      const double *__restrict__ fw, const double *__restrict__ ft,
                                                      const u32 *__restrict__ pos_nat, u64 q0) {
    extern __shared__ double smd[];
    const u32 N = 1u << logn, M = N / 2;
    const int logm = logn - 1;
    const Part pt = fft_part<SPLIT>(logn);
    const u32 v = part_row<SPLIT>();
    double *re = smd, *im = smd + pt.n;
    const u64 *mv = m + (size_t)v * N;
    // local point p receives coefficient pair k = brev(p) (bit reversal is an involution)
    for (u32 p = pt.lo + threadIdx.x; p < pt.lo + pt.n; p += blockDim.x) {
        const u32 k = __brev(p) >> (32 - logm);
        u64 a = mv[k], b = mv[k + M];
        i64 sa = a > q0 / 2 ? (i64)a - (i64)q0 : (i64)a;
        i64 sb = b > q0 / 2 ? (i64)b - (i64)q0 : (i64)b;
        double ar = __ddiv_rn((double)sa, scale), ai = __ddiv_rn((double)sb, scale);
        double tr = ft[2 * k], ti = ft[2 * k + 1];
        re[p - pt.lo] = __dsub_rn(__dmul_rn(ar, tr), __dmul_rn(ai, ti));
        im[p - pt.lo] = __dadd_rn(__dmul_rn(ar, ti), __dmul_rn(ai, tr));
    }
    __syncthreads();
    part_fft(re, im, logm, fw, false, pt);
    double *ov = out + (size_t)v * ns * nper;
    for (u32 x = threadIdx.x; x < ns * nper; x += blockDim.x) {
        u32 s = x / nper, i = x % nper;
        u32 slot = s * stride + i;
        if (slot < M) {
            const u32 p = pos_nat[slot] - pt.lo;
            if (p < pt.n) ov[x] = re[p];
        } else if (pt.lo == 0) {
            ov[x] = 0.0;
        }
    }
}

// flattened samples x[k][H*W] -> slot vectors z[ct][M]: sample k -> ct k/spc, offset (k%spc)*stride
__global__ void pack_kernel(double *z, const double *__restrict__ x, u32 nsamp, u32 spc, u32 stride, u32 len,
                            u32 M, u32 nct) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nct * M) return;
    u32 ct = (u32)(idx / M), j = (u32)(idx % M);
    u32 s = j / stride, i = j % stride;
    u32 k = ct * spc + s;
    z[idx] = (s < spc && i < len && k < nsamp) ? x[(size_t)k * len + i] : 0.0;
}

// m[b][N] = c0[b][0] + c1[b][0] * s[0]   (limb q_0, evaluation form)
__global__ void dec_combine_kernel(u64 *m, const u64 *__restrict__ ct, const u64 *__restrict__ s, u32 lp, int logn,
                                   const PrimeDev *__restrict__ pd, u32 B) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * N) return;
    u32 b = (u32)(idx >> logn), n = (u32)(idx & (N - 1));
    const PrimeDev &P = pd[0];
    const u64 *cb = ct + (size_t)b * 2 * lp * N;
    m[idx] = add_mod(cb[n], mul_mod(cb[(size_t)lp * N + n], s[n], P), P.q);
}

// c0 = u*pk0 + me ; c1 = u*pk1 + e1   (all [B][lp][N] eval; pk [2][L1][N])
__global__ void enc_combine_kernel(u64 *ct, const u64 *__restrict__ u, const u64 *__restrict__ me,
                                   const u64 *__restrict__ e1, const u64 *__restrict__ pk, u32 L1, u32 lp, int logn,
                                   const PrimeDev *__restrict__ pd, u32 B) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * lp * N) return;
    u32 n = (u32)(idx & (N - 1));
    size_t r = idx >> logn;
    u32 l = (u32)(r % lp), b = (u32)(r / lp);
    const PrimeDev &P = pd[l];
    u64 uu = u[idx];
    u64 c0 = add_mod(mul_mod(uu, pk[(size_t)l * N + n], P), me[idx], P.q);
    u64 c1 = add_mod(mul_mod(uu, pk[((size_t)L1 + l) * N + n], P), e1[idx], P.q);
    u64 *cb = ct + (size_t)b * 2 * lp * N;
    cb[(size_t)l * N + n] = c0;
    cb[((size_t)lp + l) * N + n] = c1;
}

// ------------------------------------------------------------------ host
void encode_init(Ctx *c) {
    for (const void *f : {(const void *)encode_dense_kernel<0>, (const void *)encode_dense_kernel<1>,
                          (const void *)encode_sparse_kernel<0>, (const void *)encode_sparse_kernel<1>,
                          (const void *)decode_kernel<0>, (const void *)decode_kernel<1>})
        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
}

static u32 fft_threads(u32 M) { return M >= 2048 ? 1024 : (M / 2 > 32 ? M / 2 : 32); }
// re and im of the points one CTA holds
static size_t fft_smem(const Ctx *c, int split) { return (size_t)(c->N / 2 >> split) * 16; }

static void check_err(Ctx *c) {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (h) {
        CUDA_TRY(cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream));
        throw HeError(HE_EOVERFLOW, "encoded coefficient exceeds 63 bits");
    }
}

// coefficient residues of dense slot vectors; then forward NTT.  out [nv][lp][N] eval form.
void encode_dense(Ctx *c, u64 *out, const double *z, u32 nv, double scale, u32 lp, bool check) {
    const u32 M = c->N / 2;
    double f = scale / (double)M;
    prof_begin(c);
    launch_parts(c, encode_dense_kernel<0>, encode_dense_kernel<1>, dim3(nv), ntt_min_split(c->logn), fft_threads(M >> ntt_min_split(c->logn)),
                 fft_smem(c, ntt_min_split(c->logn)), out, z, lp,
                 c->logn, f, (const double *)c->fft_w, (const double *)c->fft_t, (const u32 *)c->slot_pos_br,
                 (const PrimeDev *)c->pdev, c->err_flag);
    note_launch(c, "encode_dense");
    ntt_forward(c, out, rows_regular(nv * lp, lp, lp, 0));
    if (check) check_err(c);
}

void encode_sparse_dev(Ctx *c, u64 *out, const u32 *off, u32 nv, const u32 *pos, const double *val, u32 stride,
                       u32 ns, double scale, u32 lp, u32 ext);

// sparse slot vectors (host arrays), eval form out [nv][lp + ext][N]: limbs q_0..q_{lp-1},
// then (ext = K) the special primes, i.e. the plaintext over Q_l u P.
void encode_sparse(Ctx *c, u64 *out, const std::string &key, const std::vector<u32> &off,
                   const std::vector<u32> &pos, const std::vector<double> &val, u32 stride, u32 ns, double scale,
                   u32 lp, u32 ext) {
    const u32 M = c->N / 2;
    const u32 lpq = lp;
    lp += ext;
    u32 nv = (u32)off.size() - 1;
    std::vector<u64> h(off.size() / 2 + 1 + pos.size() / 2 + 1 + val.size() + 2, 0);
    size_t o_off = 0, o_pos = off.size() / 2 + 1, o_val = o_pos + pos.size() / 2 + 1;
    memcpy(h.data() + o_off, off.data(), off.size() * 4);
    memcpy(h.data() + o_pos, pos.data(), pos.size() * 4);
    memcpy(h.data() + o_val, val.data(), val.size() * 8);
    (void)key;
    (void)M;
    DBuf tmp(c, h.size());
    CUDA_TRY(cudaMemcpyAsync(tmp.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream));
    u64 *d = tmp.p;
    encode_sparse_dev(c, out, reinterpret_cast<const u32 *>(d + o_off), nv, reinterpret_cast<const u32 *>(d + o_pos),
                      reinterpret_cast<const double *>(d + o_val), stride, ns, scale, lpq, ext);
    check_err(c);   // also keeps the host staging vector alive until the upload is done
}

// The same from a device-resident description (no host staging and no synchronisation, so it
// can run inside a graph capture): mask v < nv covers pos/val entries [off[v], off[v+1]).
void encode_sparse_dev(Ctx *c, u64 *out, const u32 *off, u32 nv, const u32 *pos, const double *val, u32 stride,
                       u32 ns, double scale, u32 lp, u32 ext) {
    const u32 M = c->N / 2;
    const u32 lpq = lp;
    lp += ext;
    if (!nv) return;
    const double f = scale / (double)M;
    prof_begin(c);
    launch_parts(c, encode_sparse_kernel<0>, encode_sparse_kernel<1>, dim3(nv), ntt_min_split(c->logn), fft_threads(M >> ntt_min_split(c->logn)),
                 fft_smem(c, ntt_min_split(c->logn)), out, off, pos, val, stride, ns, lp, c->logn, f,
                 (const double *)c->fft_w, (const double *)c->fft_t, (const u32 *)c->slot_pos_br,
                 (const PrimeDev *)c->pdev, c->err_flag, lpq, c->L1);
    note_launch(c, "encode_sparse");
    ntt_forward(c, out, rows_regular(nv * lp, lp, lpq, c->L1));
}

void check_encode_errors(Ctx *c) { check_err(c); }

void pack_samples(Ctx *c, double *z, const double *x, u32 nsamp, u32 spc, u32 stride, u32 len, u32 nct) {
    const u32 M = c->N / 2;
    size_t total = (size_t)nct * M;
    prof_begin(c);
    pack_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(z, x, nsamp, spc, stride, len, M, nct);
    note_launch(c, "pack");
}

void enc_combine(Ctx *c, u64 *ct, const u64 *u, const u64 *me, const u64 *e1, u32 lp, u32 B) {
    size_t total = (size_t)B * lp * c->N;
    prof_begin(c);
    enc_combine_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(ct, u, me, e1, c->pk.p, c->L1, lp,
                                                                              c->logn, c->pdev, B);
    note_launch(c, "enc_combine");
}

// decrypt + decode the batch: out [B][ns][nper]
void decrypt_decode(Ctx *c, double *out, const u64 *ct, u32 B, u32 lp, double scale, u32 stride, u32 ns, u32 nper) {
    const u32 N = c->N, M = N / 2;
    DBuf m(c, (size_t)B * N);
    size_t total = (size_t)B * N;
    prof_begin(c);
    dec_combine_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(m.p, ct, c->sk.p, lp, c->logn, c->pdev,
                                                                              B);
    note_launch(c, "dec_combine");
    ntt_inverse(c, m.p, rows_regular(B, 1, 1, 0));
    prof_begin(c);
    launch_parts(c, decode_kernel<0>, decode_kernel<1>, dim3(B), ntt_min_split(c->logn), fft_threads(M >> ntt_min_split(c->logn)),
                 fft_smem(c, ntt_min_split(c->logn)), out,
                 (const u64 *)m.p, scale, stride, ns, nper, c->logn, (const double *)c->fft_w,
                 (const double *)c->fft_t, (const u32 *)c->slot_pos, c->primes[0]);
    note_launch(c, "decode");
}
