// he_internal.cuh -- shared device arithmetic and host structures of libunihenn.
//
// Residues are uint64 in [0, q) with every prime q < 2^61.  Three reductions:
//   * Shoup (Harvey 2014) for a product by a constant w with w' = floor(w*2^64/q);
//   * Barrett (Menezes et al., HAC Alg. 14.42 with base 2) for a product of two
//     variables, mu = floor(2^(2s)/q), s = bit length of q;
//   * reduce128 for a lazily accumulated 128-bit sum: (hi mod q) * (2^64 mod q)
//     by Shoup plus lo mod q by a one-word Barrett.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/unihenn.h"

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

#define HE_MAX_PRIMES 40

// ------------------------------------------------------------ device math
struct PrimeDev {
    u64 q;
    u64 mu;      // floor(2^(2s) / q)
    u64 mu64;    // floor(2^64 / q)
    u64 r64;     // 2^64 mod q
    u64 r64s;    // Shoup companion of r64
    u64 ninv;    // N^{-1} mod q
    u64 ninvs;
    u64 qneginv; // -q^{-1} mod 2^64 (Montgomery reduction)
    u32 s;       // bit length of q
    u32 pad;
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 r = a + b;
    return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a ? q - a : 0; }

// a * w mod q, w < q, ws = floor(w * 2^64 / q); any a < 2^64.
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 ws, u64 q) {
    u64 qh = mulhi64(a, ws);
    u64 r = a * w - qh * q;
    return r >= q ? r - q : r;
}

// x mod q for any 64-bit x (one-word Barrett: result of the estimate < 2q).
__device__ __forceinline__ u64 reduce64(u64 x, const PrimeDev &P) {
    u64 qh = mulhi64(x, P.mu64);
    u64 r = x - qh * P.q;
    return r >= P.q ? r - P.q : r;
}

// (hi * 2^64 + lo) mod q
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const PrimeDev &P) {
    u64 h = reduce64(hi, P);
    u64 a = mul_shoup(h, P.r64, P.r64s, P.q);
    u64 b = reduce64(lo, P);
    return add_mod(a, b, P.q);
}

// Montgomery reduction (Montgomery 1985) of a 128-bit x = hi*2^64 + lo < q*2^64:
// x * 2^{-64} mod q in [0, q).  m = lo * (-q^{-1}) makes x + m*q divisible by 2^64.
__device__ __forceinline__ u64 redc128(u64 lo, u64 hi, const PrimeDev &P) {
    const u64 m = lo * P.qneginv;
    const u64 t = hi + mulhi64(m, P.q) + (lo != 0 ? 1 : 0);
    return t >= P.q ? t - P.q : t;
}

// asynchronous 8-byte global -> shared copies (cp.async, grouped with commit / wait)
__device__ __forceinline__ void cp_async8(u64 *smem, const u64 *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// bulk prefetch of a contiguous global region into L2 (one instruction, TMA unit);
// address 16-byte aligned, size a multiple of 16 bytes
__device__ __forceinline__ void l2_prefetch_bulk(const void *gmem, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// a * b mod q for a, b < q (HAC 14.42, base 2, k = s)
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeDev &P) {
    u64 lo = a * b;
    u64 hi = mulhi64(a, b);
    u32 s = P.s;
    u64 q1 = (hi << (65 - s)) | (lo >> (s - 1));
    u64 t_lo = q1 * P.mu;
    u64 t_hi = mulhi64(q1, P.mu);
    u64 q3 = (t_hi << (63 - s)) | (t_lo >> (s + 1));
    u64 r = lo - q3 * P.q;
    if (r >= P.q) r -= P.q;
    if (r >= P.q) r -= P.q;
    return r;
}

// 128-bit accumulator
struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void mac128(Acc128 &acc, u64 a, u64 b) {
    const u64 plo = a * b;
    const u64 phi = mulhi64(a, b);
    // 128-bit add through the carry flag (add.cc / addc) rather than a compare
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, %3;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(plo), "l"(phi));
}

__device__ __forceinline__ u32 brev_bits(u32 x, int bits) { return __brev(x) >> (32 - bits); }

// index in bit-reversed evaluation order whose value sigma_g takes for slot i:
// slot i holds a(psi^(2*brev(i)+1)); sigma_g(a) there equals a(psi^(g*(2*brev(i)+1))).
__device__ __forceinline__ u32 galois_src(u32 i, u32 g, int logn) {
    u32 e = 2 * brev_bits(i, logn) + 1;
    u32 m = (u32)(((u64)g * e) & ((2ull << logn) - 1));
    return brev_bits((m - 1) >> 1, logn);
}

// SplitMix64 (Steele, Lea & Flood 2014; variant-13 finaliser), counter-based:
// word i of stream `st` under `seed` = output #i of a SplitMix64 seeded with
// output #st of a SplitMix64 seeded with `seed`.
__host__ __device__ __forceinline__ u64 sm64_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ u64 sm64_state(u64 seed, u64 stream) {
    return sm64_mix(seed + (stream + 1) * 0x9e3779b97f4a7c15ULL);
}
__host__ __device__ __forceinline__ u64 sm64_word(u64 state, u64 i) {
    return sm64_mix(state + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

// randomness stream ids: purpose<<56 | key_id<<32 | digit<<16 | limb
enum { RS_SK = 1, RS_PK_A = 2, RS_PK_E = 3, RS_KSK_A = 4, RS_KSK_E = 5, RS_ENC_U = 6, RS_ENC_E0 = 7, RS_ENC_E1 = 8 };
__host__ __device__ __forceinline__ u64 stream_id(u64 purpose, u64 key, u64 digit, u64 limb) {
    return (purpose << 56) | (key << 32) | (digit << 16) | limb;
}

// ------------------------------------------------------------ host side
struct HeError : std::runtime_error {
    he_status code;
    HeError(he_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define CUDA_TRY(x)                                                                      \
    do {                                                                                 \
        cudaError_t e__ = (x);                                                           \
        if (e__ != cudaSuccess)                                                          \
            throw HeError(e__ == cudaErrorMemoryAllocation ? HE_ENOMEM : HE_ECUDA,       \
                          std::string(#x) + ": " + cudaGetErrorString(e__));             \
    } while (0)

struct Ctx;
void prof_begin(Ctx *c);                                        // start event of the next launch (profiling)
// set while this thread captures a CUDA graph: no device-wide synchronisation then
void set_capturing(bool on);
// error check, launch counter, end event; bytes = algorithmic bytes, ops = algorithmic primitive
// operations of the launch (NTT butterflies or 64x64->128 multiply-accumulates)
void note_launch(Ctx *c, const char *what, double bytes = 0, double ops = 0);

// Caching device allocator: buffers are returned to per-size free lists and
// reused in stream order (all work of a context runs on one stream), so the
// steady state of an inference issues no cudaMalloc/cudaFree.
struct Pool {
    std::map<size_t, std::vector<void *>> free_;
    std::map<void *, size_t> size_;
    size_t bytes_live = 0, bytes_cached = 0;
    // a compiled model's graph pool: a request takes the smallest cached block of at least
    // its size (not only an exact size), so the model's graphs, which never run
    // concurrently, hold the largest batch shape's buffers once for every shape; and its
    // cached blocks are never freed while the model lives (captured graphs refer to them)
    bool graph = false;
    void *get(size_t bytes);
    void put(void *p);
    void release_cached();
    void release_all();
};

// A device buffer owned through the pool
struct DBuf {
    Pool *pool = nullptr;
    u64 *p = nullptr;
    size_t words = 0;
    DBuf() = default;
    DBuf(Ctx *c, size_t w);
    ~DBuf();
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : pool(o.pool), p(o.p), words(o.words) { o.p = nullptr; o.words = 0; }
    DBuf &operator=(DBuf &&o) noexcept;
};

// slot layout of a ciphertext (paper Sec. III-A/B, IV, V)
struct Layout {
    u32 W_img = 0, H_img = 0;   // original row pitch / height
    u32 W = 0, H = 0;           // current valid width/height
    u32 I = 1;                  // interval
    u32 stride = 0;             // slots per sample
    u32 n_samples = 1;          // sample positions in masks
    u32 dims = 2;               // 2-D image or 1-D signal
    double pending = 1.0;       // deferred pooling factor
    int prev = 0;               // 0 input, 1 conv, 2 avgpool, 3 flatten, 4 fc
    u32 D = 0;                  // flattened length
    u32 C = 1;                  // input channels in one ciphertext (channel i at i*W_img*H_img)
};
enum { PREV_INPUT = 0, PREV_CONV = 1, PREV_POOL = 2, PREV_FLAT = 3, PREV_FC = 4 };

// knobs of the autotuner (tune.cu): launch shapes that change speed, never results
enum {
    TUNE_NTT = 0,      // split limbs over 2-CTA clusters: 0 / 1
    TUNE_MODDOWN,      // the same for the fused ModDown kernel
    TUNE_RESCALE,      // the same for the fused rescale kernel
    TUNE_MAC_GROUP,    // outputs per MAC launch (accumulators held in registers)
    TUNE_LAZY_BT,      // ciphertexts per thread in the hoisted key-switch accumulation
    TUNE_LAZY_ORDER,   // its grid order: 0 coefficient tiles fastest, 1 ciphertext groups fastest
    TUNE_MAC_BK,       // polynomials per MAC CTA (the rest of its 256 threads cover coefficients)
    TUNE_MAC_SPLIT,    // threads per coefficient sharing a MAC group of 7..12 outputs: 1 / 2
    TUNE_COMB_BT,      // ciphertexts per thread of the one-pass combination (ks_comb): 2 / 4
    TUNE_COMB_FOLD,    // ciphertexts from which a one-channel weighted combination folds its weights into the keys
    TUNE_MAC_TC,       // MAC of 6+ outputs: limbs of at most this many bytes on the tensor cores (0 none, default / 5 / 8)
    TUNE_COUNT
};

struct Ctx : std::enable_shared_from_this<Ctx> {
    // Serialises host-side use of the context (pools, table cache, stream order of
    // multi-launch operations) between threads: every C entry point and the
    // serving loop hold it while they enqueue work or release buffers.
    std::recursive_mutex mu;
    int tuned[TUNE_COUNT] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};   // -1: default
    // parameters
    int logn = 0;
    u32 N = 0, L1 = 0, K = 0, dnum = 0, alpha = 0;
    double scale = 0;
    u64 seed = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<u64> primes;       // L1 data then K special
    std::vector<u64> psi;
    std::vector<PrimeDev> pdev_h;
    // device tables
    PrimeDev *pdev = nullptr;      // [nprimes]
    u64 *tw = nullptr;             // per prime (4N words): (psi_rev, Shoup) pairs, then (ipsi_rev, Shoup) pairs
    double *fft_w = nullptr;       // cos/sin of 2*pi*k/M, k < M/2 (interleaved)
    double *fft_t = nullptr;       // cos/sin of pi*k/N, k < M (interleaved)
    u32 *slot_pos_br = nullptr;    // bit-reversed DFT position of slot j
    u32 *slot_pos = nullptr;       // DFT position of slot j
    Pool pool;
    Pool *active = nullptr;        // pool that new buffers come from (a model's private pool during graph capture)
    // keys
    bool have_keys = false;
    bool naf = false;              // power-of-two Galois keys only: rotations by non-adjacent-form chains
    // paper-order schedule (he_context_set_schedule): every rotation its own key switch, masks
    // multiplied over Q_l after the rotation, the centred rescale; no hoisted combination
    bool literal = false;
    DBuf sk;                       // [L1+K][N] eval
    DBuf pk;                       // [2][L1][N]
    DBuf rlk;                      // [dnum][2][L1+K][N]
    std::map<u32, DBuf> gk;        // Galois element -> key [dnum][2][L+1+K][N]
    std::map<u32, DBuf> gkp;       // the same keys permuted by sigma_g^{-1}
    // per-level constant tables (host-built, device-resident)
    std::map<std::string, DBuf> cache;
    uint64_t launches = 0;
    // per-launch CUDA-event profiling (he_profile_begin / he_profile_end)
    struct ProfRec {
        const char *name;
        double bytes, ops;
        cudaEvent_t a, b;
        std::string tag;
    };
    bool profiling = false;
    std::string prof_tag;          // e.g. the layer being evaluated
    cudaEvent_t prof_start = nullptr;
    std::vector<cudaEvent_t> ev_free;
    std::vector<ProfRec> recs;
    cudaEvent_t new_event();
    int *err_flag = nullptr;       // device error word (encoder overflow etc.)

    u32 nprimes() const { return L1 + K; }
    u64 *tw_fwd(u32 p) const { return tw + (size_t)p * 4 * N; }
    u32 galois_elt(int64_t step) const;
    u32 galois_inverse(u32 g) const;
    u64 *const_table(const std::string &key, const std::vector<u64> &host);
};

// ---- kernels / ops (defined across the .cu files)
// ntt.cu
struct RowSet {         // rows of N words: row r at base + off(r)*N, prime pidx(r)
    const u32 *list;    // packed (limb_offset << 8 | prime), or nullptr for the regular form
    u32 n;
    u32 period, lp, pbase;   // regular form: row r -> offset r, prime (r%period<lp ? r%period : pbase + r%period - lp)
};
void ntt_forward(Ctx *c, u64 *base, const RowSet &rs);
void ntt_inverse(Ctx *c, u64 *base, const RowSet &rs);
// the inner launch of the two-kernel NTT over the rows of rs (ntt_block.cuh)
void ntt2_inner(Ctx *c, u64 *base, const RowSet &rs, int inverse);
// dst [B][lp][N] = inverse NTT of limbs 0..lp-1 of B polynomials at src, batch stride src_bstride;
// true when the rows were also copied to the ModUp digits' own rows of own [B][beta][E][N]
bool ntt_inverse_from(Ctx *c, u64 *dst, const u64 *src, size_t src_bstride, u32 B, u32 lp, u64 *own = nullptr,
                      u32 beta = 0, u32 E = 0);
RowSet rows_regular(u32 n, u32 period, u32 lp, u32 pbase);
RowSet rows_list(Ctx *c, const std::string &key, const std::vector<u32> &packed);

// keyswitch.cu, he.cu, layers.cu: see the respective files
std::string fmt(const char *f, ...);

// holds a context's lock for the enclosing scope
struct CtxLock {
    std::lock_guard<std::recursive_mutex> g;
    explicit CtxLock(Ctx *c) : g(c->mu) {}
};

// a tuned knob, or dflt when it was not tuned
static inline int tune_get(const Ctx *c, int knob, int dflt) { return c->tuned[knob] >= 0 ? c->tuned[knob] : dflt; }
// limb layout of an NTT-carrying kernel family (TUNE_NTT / TUNE_MODDOWN / TUNE_RESCALE):
// 0 one CTA per limb, 1 a 2-CTA cluster per limb, NTT_TWO_KERNEL an outer launch over columns
// and an inner launch over 1024-coefficient blocks (ntt_block.cuh); tuned, else the default
// for N (two-kernel from 2^14 up), never a layout N does not allow
#define NTT_TWO_KERNEL 2
int ntt_layout(const Ctx *c, int knob);
