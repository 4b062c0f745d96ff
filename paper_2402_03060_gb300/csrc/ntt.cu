// ntt.cu -- batched negacyclic NTT / inverse NTT over sets of limbs.
// One CTA per limb (row of N words), or a cluster of two CTAs per limb above
// N = 2^14; the limb is staged in shared memory (N*8 bytes: 128 KiB at
// N = 16384), transformed with part_ntt_* and written back.
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

static void ntt_launch(Ctx *c, u64 *base, const RowSet &rs, int inverse) {
    if (rs.n == 0) return;
    prof_begin(c);
    const int sp = tune_split(c, TUNE_NTT);
    launch_parts(c, ntt_rows_kernel<0>, ntt_rows_kernel<1>, dim3(rs.n), sp, ntt_part_threads(c->logn, sp), ntt_part_smem(c->logn, sp), base, rs,
                 (const u64 *)c->tw, (const PrimeDev *)c->pdev, c->logn, inverse);
    // each limb read and written once; (N/2) log2 N butterflies per limb
    note_launch(c, inverse ? "intt" : "ntt", 16.0 * rs.n * c->N, (double)rs.n * (c->N / 2) * c->logn);
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
