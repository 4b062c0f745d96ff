// ntt.cu -- batched negacyclic NTT / inverse NTT over sets of limbs, in the limb layout the
// context uses (ntt_layout): one CTA per limb (row of N words) or a cluster of two CTAs per
// limb, the limb staged in shared memory (N*8 bytes: 128 KiB at N = 16384) and transformed
// with part_ntt_*; or the two-kernel form of ntt_block.cuh (outer stages over the 1024
// columns, inner stages over 1024-coefficient blocks), the default from N = 2^14.
#include "ntt_block.cuh"

__device__ __forceinline__ void row_of(const RowSet &rs, u32 r, u32 &off, u32 &prime) {
    if (rs.list) {
        u32 v = rs.list[r];
        off = v >> 8;
        prime = v & 0xff;
    } else {
        off = r;
        u32 w = r % rs.period;
        prime = w < rs.lp ? w : rs.pbase + (w - rs.lp);
    }
}

template <int SPLIT>
__global__ void __launch_bounds__(NTT_MAX_THREADS) ntt_rows_kernel(u64 *base, RowSet rs, const u64 *tw_all,
                                                        const PrimeDev *pd, int logn, int inverse) {
    extern __shared__ u64 sm[];
    const u32 N = 1u << logn;
    const Part pt = ntt_part<SPLIT>(logn);
    u32 off, prime;
    row_of(rs, part_row<SPLIT>(), off, prime);
    u64 *g = base + (size_t)off * N + pt.lo;
    const u64 *tw = tw_all + (size_t)prime * 4 * N;
    const PrimeDev P = pd[prime];
    block_load(sm, g, pt.n);
    if (inverse)
        part_ntt_inv(sm, pt, logn, tw, P.q, P.ninv, P.ninvs);
    else
        part_ntt_fwd(sm, pt, logn, tw, P.q);
    block_store(g, sm, pt.n);
}

// two-kernel form (ntt_block.cuh): the outer stages of every row, one column per thread
template <int R>
__global__ void __launch_bounds__(NTT2_COLS) ntt2_outer_kernel(u64 *base, RowSet rs, const u64 *tw_all,
                                                               const PrimeDev *pd, int inverse) {
    const u32 N = 1024u << R;
    u32 off, prime;
    row_of(rs, blockIdx.x, off, prime);
    u64 *col = base + (size_t)off * N + blockIdx.y * NTT2_COLS + threadIdx.x;
    const u64 *tw = tw_all + (size_t)prime * 4 * N;
    const PrimeDev P = pd[prime];
    u64 v[1 << R];
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) v[k] = col[1024u * k];
    if (inverse)
        outer_inv_regs<R>(v, tw, N, P.q, P.ninv, P.ninvs);
    else
        outer_fwd_regs<R>(v, tw, P.q);
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) col[1024u * k] = v[k];
}

// ... and the inner stages of every 1024-coefficient block (grid.x = rows, grid.y = blocks)
__global__ void __launch_bounds__(NTT2_INNER_THREADS) ntt2_inner_kernel(u64 *base, RowSet rs, const u64 *tw_all,
                                                                        const PrimeDev *pd, int logn, int inverse) {
    __shared__ u64 sm[1024 + 1024 / 16];
    const u32 N = 1u << logn;
    u32 off, prime;
    row_of(rs, blockIdx.x, off, prime);
    const u32 goff = 1024u * blockIdx.y;
    u64 *g = base + (size_t)off * N + goff;
    const u64 *tw = tw_all + (size_t)prime * 4 * N;
    const u64 q = pd[prime].q;
    block_load(sm, g, 1024);
    if (inverse)
        inner_inv_block(sm, logn, tw, q, goff);
    else
        inner_fwd_block(sm, logn, tw, q, goff);
    block_store(g, sm, 1024);
}

// the inner launch of the two-kernel form over the rows of rs (forward after, inverse before the outer one)
void ntt2_inner(Ctx *c, u64 *base, const RowSet &rs, int inverse) {
    ntt2_inner_kernel<<<dim3(rs.n, c->N >> NTT2_INNER_LOGN), NTT2_INNER_THREADS, 0, c->stream>>>(
        base, rs, (const u64 *)c->tw, (const PrimeDev *)c->pdev, c->logn, inverse);
}

// inner inverse stages of rows read from a strided source: row r = b*lp + t of dst (prime t) is
// limb t of ciphertext b at src + b*src_bstride + t*N (the c1 rows of a ciphertext batch, say).
// With own: each row is also copied as read to the ModUp digits' own row, D[b][t/alpha][t] of
// D [B][beta][E][N].
__global__ void __launch_bounds__(NTT2_INNER_THREADS) ntt2_inner_inv_from_kernel(u64 *dst, const u64 *__restrict__ src,
                                                                                 size_t src_bstride, u32 lp,
                                                                                 u64 *own, u32 alpha, u32 beta,
                                                                                 u32 E, const u64 *tw_all,
                                                                                 const PrimeDev *pd, int logn) {
    __shared__ u64 sm[1024 + 1024 / 16];
    const u32 N = 1u << logn;
    const u32 r = blockIdx.x, b = r / lp, t = r % lp;
    const u32 goff = 1024u * blockIdx.y;
    const ulonglong2 *g2 = reinterpret_cast<const ulonglong2 *>(src + (size_t)b * src_bstride + (size_t)t * N + goff);
    ulonglong2 *o2 =
        own ? reinterpret_cast<ulonglong2 *>(own + (((size_t)b * beta + t / alpha) * E + t) * N + goff) : nullptr;
    for (u32 k = threadIdx.x; k < 512; k += blockDim.x) {
        const ulonglong2 v = g2[k];
        sm[spad(2 * k)] = v.x;
        sm[spad(2 * k + 1)] = v.y;
        if (o2) o2[k] = v;
    }
    __syncthreads();
    inner_inv_block(sm, logn, tw_all + (size_t)t * 4 * N, pd[t].q, goff);
    block_store(dst + (size_t)r * N + goff, sm, 1024);
}

// dst [B][lp][N] = inverse NTT of limbs 0..lp-1 of the B ciphertext polynomials at src (batch
// stride src_bstride words): the two-kernel form reads the rows where they are (and, with own,
// copies them to the ModUp digits' own rows of own [B][beta][E][N]: returns true); the other
// layouts copy them first (returns false: own untouched)
bool ntt_inverse_from(Ctx *c, u64 *dst, const u64 *src, size_t src_bstride, u32 B, u32 lp, u64 *own, u32 beta,
                      u32 E) {
    const RowSet rs = rows_regular(B * lp, lp, lp, 0);
    if (ntt_layout(c, TUNE_NTT) != NTT_TWO_KERNEL) {
        CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)lp * c->N * 8, src, src_bstride * 8, (size_t)lp * c->N * 8, B,
                                   cudaMemcpyDeviceToDevice, c->stream));
        ntt_inverse(c, dst, rs);
        return false;
    }
    if (rs.n == 0) return own != nullptr;
    if (rs.n > 0x7fffffffu) throw HeError(HE_EINVAL, "NTT: too many rows");
    const double bytes = 16.0 * rs.n * c->N, bfly = (double)rs.n * (c->N / 2);
    prof_begin(c);
    ntt2_inner_inv_from_kernel<<<dim3(rs.n, c->N >> NTT2_INNER_LOGN), NTT2_INNER_THREADS, 0, c->stream>>>(
        dst, src, src_bstride, lp, own, c->alpha, beta, E, (const u64 *)c->tw, (const PrimeDev *)c->pdev, c->logn);
    note_launch(c, "intt", bytes / 2 + (own ? 8.0 * rs.n * c->N : 0.0), bfly * NTT2_INNER_LOGN);
    prof_begin(c);
    NTT2_OUTER_LAUNCH(c, ntt2_outer_kernel, c->logn, rs.n, dst, rs, (const u64 *)c->tw, (const PrimeDev *)c->pdev, 1);
    note_launch(c, "intt", bytes / 2, bfly * (c->logn - NTT2_INNER_LOGN));
    return own != nullptr;
}

static void ntt_launch(Ctx *c, u64 *base, const RowSet &rs, int inverse) {
    if (rs.n == 0) return;
    if (rs.n > 0x7fffffffu) throw HeError(HE_EINVAL, "NTT: too many rows");
    const char *name = inverse ? "intt" : "ntt";
    // each limb read and written once; (N/2) log2 N butterflies per limb
    const double bytes = 16.0 * rs.n * c->N, bfly = (double)rs.n * (c->N / 2);
    const int sp = ntt_layout(c, TUNE_NTT);
    if (sp == NTT_TWO_KERNEL) {
        // the algorithmic bytes split evenly, the butterflies by stage count (10 inner, logn - 10 outer)
        auto inner = [&] {
            prof_begin(c);
            ntt2_inner(c, base, rs, inverse);
            note_launch(c, name, bytes / 2, bfly * NTT2_INNER_LOGN);
        };
        if (inverse) inner();
        prof_begin(c);
        NTT2_OUTER_LAUNCH(c, ntt2_outer_kernel, c->logn, rs.n, base, rs, (const u64 *)c->tw,
                          (const PrimeDev *)c->pdev, inverse);
        note_launch(c, name, bytes / 2, bfly * (c->logn - NTT2_INNER_LOGN));
        if (!inverse) inner();
        return;
    }
    prof_begin(c);
    launch_parts(c, ntt_rows_kernel<0>, ntt_rows_kernel<1>, dim3(rs.n), sp, ntt_part_threads(c->logn, sp),
                 ntt_part_smem(c->logn, sp), base, rs, (const u64 *)c->tw, (const PrimeDev *)c->pdev, c->logn,
                 inverse);
    note_launch(c, name, bytes, bfly * c->logn);
}

void ntt_forward(Ctx *c, u64 *base, const RowSet &rs) { ntt_launch(c, base, rs, 0); }
void ntt_inverse(Ctx *c, u64 *base, const RowSet &rs) { ntt_launch(c, base, rs, 1); }

RowSet rows_regular(u32 n, u32 period, u32 lp, u32 pbase) {
    RowSet r;
    r.list = nullptr;
    r.n = n;
    r.period = period;
    r.lp = lp;
    r.pbase = pbase;
    return r;
}

RowSet rows_list(Ctx *c, const std::string &key, const std::vector<u32> &packed) {
    RowSet r;
    r.n = (u32)packed.size();
    r.period = 1;
    r.lp = 1;
    r.pbase = 0;
    std::vector<u64> h((packed.size() + 1) / 2 + 1, 0);
    memcpy(h.data(), packed.data(), packed.size() * sizeof(u32));
    r.list = reinterpret_cast<const u32 *>(c->const_table("rows:" + key, h));
    return r;
}

void ntt_init_attrs(Ctx *c) {
    (void)c;
    CUDA_TRY(cudaFuncSetAttribute(ntt_rows_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    CUDA_TRY(cudaFuncSetAttribute(ntt_rows_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
}
