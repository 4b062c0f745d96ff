// he.cu -- context, device memory pool, key generation, encryption and the
// ciphertext operations (Add, Mul (P), Mul (C), Rot of paper Sec. II-B) over
// batches of ciphertexts.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "ntt_block.cuh"
#include "ops.cuh"

std::string fmt(const char *f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}

cudaEvent_t Ctx::new_event() {
    if (!ev_free.empty()) {
        cudaEvent_t e = ev_free.back();
        ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    return e;
}

void prof_begin(Ctx *c) {
    if (!c->profiling) return;
    c->prof_start = c->new_event();
    CUDA_TRY(cudaEventRecord(c->prof_start, c->stream));
}

void note_launch(Ctx *c, const char *what, double bytes, double ops) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw HeError(HE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (c->profiling && c->prof_start) {
        cudaEvent_t b = c->new_event();
        CUDA_TRY(cudaEventRecord(b, c->stream));
        c->recs.push_back({what, bytes, ops, c->prof_start, b, c->prof_tag});
        c->prof_start = nullptr;
    }
}

// ------------------------------------------------------------------ pool
static thread_local bool tl_capturing = false;
void set_capturing(bool on) { tl_capturing = on; }

void *Pool::get(size_t bytes) {
    bytes = (bytes + 4095) & ~(size_t)4095;
    if (bytes == 0) bytes = 4096;
    auto it = free_.find(bytes);
    if (graph)
        for (it = free_.lower_bound(bytes); it != free_.end() && it->second.empty(); ++it) {
        }
    void *p = nullptr;
    if (it != free_.end() && !it->second.empty()) {
        p = it->second.back();
        it->second.pop_back();
        bytes = it->first;   // the block's own size
        bytes_cached -= bytes;
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            // give cached blocks back and retry once -- not a graph pool's (captured graphs
            // use them) and not during a capture (the release synchronises the device)
            if (graph || tl_capturing) throw HeError(HE_ENOMEM, fmt("device allocation of %zu bytes failed", bytes));
            release_cached();
            e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw HeError(HE_ENOMEM, fmt("device allocation of %zu bytes failed", bytes));
            }
        }
        size_[p] = bytes;
    }
    bytes_live += bytes;
    return p;
}

void Pool::put(void *p) {
    if (!p) return;
    auto sz = size_.find(p);
    if (sz == size_.end()) return;   // not from this pool (already released)
    size_t bytes = sz->second;
    free_[bytes].push_back(p);
    bytes_live -= bytes;
    bytes_cached += bytes;
}

void Pool::release_cached() {
    cudaDeviceSynchronize();
    for (auto &kv : free_) {
        for (void *p : kv.second) {
            cudaFree(p);
            size_.erase(p);
        }
        kv.second.clear();
    }
    bytes_cached = 0;
}

void Pool::release_all() {
    release_cached();
    for (auto &kv : size_) cudaFree(kv.first);
    size_.clear();
    bytes_live = 0;
}

DBuf::DBuf(Ctx *c, size_t w) : words(w) {
    pool = c->active ? c->active : &c->pool;
    p = (u64 *)pool->get(w * 8);
}
DBuf::~DBuf() {
    if (p && pool) pool->put(p);
}
DBuf &DBuf::operator=(DBuf &&o) noexcept {
    if (this != &o) {
        if (p && pool) pool->put(p);
        pool = o.pool;
        p = o.p;
        words = o.words;
        o.p = nullptr;
        o.words = 0;
    }
    return *this;
}

u64 *Ctx::const_table(const std::string &key, const std::vector<u64> &host) {
    auto it = cache.find(key);
    if (it != cache.end()) return it->second.p;
    Pool *saved = active;   // tables always live in the context's own pool
    active = nullptr;
    DBuf b(this, host.size() ? host.size() : 1);
    active = saved;
    if (!host.empty())
        CUDA_TRY(cudaMemcpyAsync(b.p, host.data(), host.size() * 8, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));   // host vector may go away
    u64 *p = b.p;
    cache.emplace(key, std::move(b));
    return p;
}

// g^{-1} mod 2N: the odd residues mod 2N form a group of order N, so g^{-1} = g^{N-1}
u32 Ctx::galois_inverse(u32 g) const {
    const u64 twoN = 2ull * N;
    u64 r = 1, b = g, e = N - 1;
    while (e) {
        if (e & 1) r = r * b % twoN;
        b = b * b % twoN;
        e >>= 1;
    }
    return (u32)r;
}

u32 Ctx::galois_elt(int64_t step) const {
    const u64 M = N / 2, twoN = 2ull * N;
    u64 e = (u64)(((step % (int64_t)M) + (int64_t)M) % (int64_t)M);
    u64 r = 1, b = 5;
    while (e) {
        if (e & 1) r = r * b % twoN;
        b = b * b % twoN;
        e >>= 1;
    }
    return (u32)r;
}

// ------------------------------------------------------------------ number theory
static u64 mulm(u64 a, u64 b, u64 q) { return (u64)((unsigned __int128)a * b % q); }
static u64 powm(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulm(r, a, q);
        a = mulm(a, a, q);
        e >>= 1;
    }
    return r;
}
// deterministic Miller-Rabin for 64-bit integers (bases: the first 12 primes)
static bool prime64(u64 n) {
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    for (u64 a : bases) {
        u64 x = powm(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = mulm(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

static std::vector<u64> chain_primes(const std::vector<u32> &bits, int logn) {
    const u64 m = 2ull << logn;
    std::vector<u64> out;
    for (u32 b : bits) {
        u64 top = (b >= 64) ? ~0ull : ((1ull << b) - 1);
        u64 c = top / m * m + 1;
        if (c > top) c -= m;
        bool found = false;
        for (; c > m; c -= m) {
            if (std::find(out.begin(), out.end(), c) != out.end()) continue;
            if (prime64(c)) {
                found = true;
                break;
            }
        }
        if (!found) throw HeError(HE_EINVAL, fmt("no %u-bit prime = 1 mod 2N", b));
        out.push_back(c);
    }
    return out;
}

// smallest primitive 2N-th root of unity mod q
static u64 min_root(u64 q, int logn) {
    const u64 n = 1ull << logn, m = 2 * n;
    u64 root = 0;
    for (u64 g = 2; g < (1u << 20); ++g) {
        u64 r = powm(g, (q - 1) / m, q);
        if (powm(r, n, q) == q - 1) {
            root = r;
            break;
        }
    }
    if (!root) throw HeError(HE_EINVAL, "no primitive root");
    u64 best = root, x = root, r2 = mulm(root, root, q);
    for (u64 k = 1; k < n; ++k) {
        x = mulm(x, r2, q);
        if (x < best) best = x;
    }
    return best;
}

static u32 bitrev(u32 x, int bits) {
    u32 r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

// ------------------------------------------------------------------ context
void ntt_init_attrs(Ctx *c);
void keyswitch_init(Ctx *c);
void mac_init(Ctx *c);

Ctx *ctx_create(const he_params *p) {
    if (!p || p->log2n < 4 || p->log2n > 15 || p->n_data < 1 || p->n_data > 32 || p->n_special < 1 ||
        p->n_special > 4 || !p->prime_bits || p->dnum < 1 || p->dnum > p->n_data || p->dnum > 16)
        throw HeError(HE_EINVAL, "he_params out of range");
    if (p->n_data + p->n_special > HE_MAX_PRIMES) throw HeError(HE_EINVAL, "too many primes");
    std::vector<u32> bits(p->prime_bits, p->prime_bits + p->n_data + p->n_special);
    for (u32 b : bits)
        if (b < 20 || b > 60) throw HeError(HE_EINVAL, "prime bit sizes must be within 20..60");
    std::unique_ptr<Ctx> c(new Ctx());
    c->logn = (int)p->log2n;
    c->N = 1u << p->log2n;
    c->L1 = p->n_data;
    c->K = p->n_special;
    c->dnum = p->dnum;
    c->alpha = (c->L1 + c->dnum - 1) / c->dnum;
    if (c->alpha > 8) throw HeError(HE_EINVAL, "digits of more than 8 data primes are not supported (raise dnum)");
    c->scale = std::pow(2.0, p->log2_scale);
    c->seed = p->seed;
    c->device = p->device;
    CUDA_TRY(cudaSetDevice(c->device));
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    c->primes = chain_primes(bits, c->logn);
    const u32 N = c->N, M = N / 2, np = c->nprimes();
    // prime constants
    for (u32 i = 0; i < np; ++i) {
        u64 q = c->primes[i];
        c->psi.push_back(min_root(q, c->logn));
        PrimeDev d;
        memset(&d, 0, sizeof d);
        d.q = q;
        u32 s = 64 - __builtin_clzll(q);
        d.s = s;
        d.mu = (u64)(((unsigned __int128)1 << (2 * s)) / q);
        d.mu64 = (u64)((((unsigned __int128)1) << 64) / q);
        d.r64 = (u64)((((unsigned __int128)1) << 64) % q);
        d.r64s = (u64)(((unsigned __int128)d.r64 << 64) / q);
        {
            u64 inv = q;   // Newton iteration for q^{-1} mod 2^64 (q odd): 5 steps double 3 correct bits to 96
            for (int it = 0; it < 5; ++it) inv *= 2 - q * inv;
            d.qneginv = (u64)0 - inv;
        }
        d.ninv = powm(N % q, q - 2, q);
        d.ninvs = (u64)(((unsigned __int128)d.ninv << 64) / q);
        c->pdev_h.push_back(d);
    }
    CUDA_TRY(cudaMalloc(&c->pdev, sizeof(PrimeDev) * np));
    CUDA_TRY(cudaMemcpy(c->pdev, c->pdev_h.data(), sizeof(PrimeDev) * np, cudaMemcpyHostToDevice));
    // NTT twiddles
    std::vector<u64> tw((size_t)np * 4 * N);
    for (u32 i = 0; i < np; ++i) {
        u64 q = c->primes[i], psi = c->psi[i], ipsi = powm(psi, q - 2, q);
        u64 *t = tw.data() + (size_t)i * 4 * N;
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (u32 k = 1; k < N; ++k) {
            pw[k] = mulm(pw[k - 1], psi, q);
            ipw[k] = mulm(ipw[k - 1], ipsi, q);
        }
        for (u32 k = 0; k < N; ++k) {   // (w, w') pairs, forward then inverse
            u64 w = pw[bitrev(k, c->logn)], iw = ipw[bitrev(k, c->logn)];
            t[2 * k] = w;
            t[2 * k + 1] = (u64)(((unsigned __int128)w << 64) / q);
            t[2 * N + 2 * k] = iw;
            t[2 * N + 2 * k + 1] = (u64)(((unsigned __int128)iw << 64) / q);
        }
    }
    CUDA_TRY(cudaMalloc(&c->tw, tw.size() * 8));
    CUDA_TRY(cudaMemcpy(c->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));
    // FFT tables: w_k = exp(2*pi*i*k/M) (k < M/2), twist zeta^k = exp(i*pi*k/N) (k < M)
    std::vector<double> fw(M), ft(2 * (size_t)M);
    for (u32 k = 0; k < M / 2; ++k) {
        double ang = 2.0 * M_PI * (double)k / (double)M;
        fw[2 * k] = cos(ang);
        fw[2 * k + 1] = sin(ang);
    }
    for (u32 k = 0; k < M; ++k) {
        double ang = M_PI * (double)k / (double)N;
        ft[2 * k] = cos(ang);
        ft[2 * k + 1] = sin(ang);
    }
    CUDA_TRY(cudaMalloc(&c->fft_w, fw.size() * 8 + 8));
    CUDA_TRY(cudaMemcpy(c->fft_w, fw.data(), fw.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&c->fft_t, ft.size() * 8));
    CUDA_TRY(cudaMemcpy(c->fft_t, ft.data(), ft.size() * 8, cudaMemcpyHostToDevice));
    // slot j <-> DFT index (5^j mod 2N - 1)/4, natural and bit-reversed
    std::vector<u32> pos(M), posbr(M);
    u64 t5 = 1;
    for (u32 j = 0; j < M; ++j) {
        u32 s = (u32)((t5 - 1) / 4);
        pos[j] = s;
        posbr[j] = bitrev(s, c->logn - 1);
        t5 = t5 * 5 % (2ull * N);
    }
    CUDA_TRY(cudaMalloc(&c->slot_pos, M * 4));
    CUDA_TRY(cudaMemcpy(c->slot_pos, pos.data(), M * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&c->slot_pos_br, M * 4));
    CUDA_TRY(cudaMemcpy(c->slot_pos_br, posbr.data(), M * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&c->err_flag, sizeof(int)));
    CUDA_TRY(cudaMemset(c->err_flag, 0, sizeof(int)));
    ntt_init_attrs(c.get());
    keyswitch_init(c.get());
    mac_tc_init();
    mac_init(c.get());
    encode_init(c.get());
    return c.release();
}

void ctx_destroy(Ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    c->sk = DBuf();
    c->pk = DBuf();
    c->rlk = DBuf();
    c->gk.clear();
    c->gkp.clear();
    c->cache.clear();
    c->pool.release_all();
    cudaFree(c->pdev);
    cudaFree(c->tw);
    cudaFree(c->fft_w);
    cudaFree(c->fft_t);
    cudaFree(c->slot_pos);
    cudaFree(c->slot_pos_br);
    cudaFree(c->err_flag);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ------------------------------------------------------------------ keys
// out[t][n] += cst[t] * x[t][n] for rows t in [lo, hi) (cst Shoup pairs)
__global__ void add_scaled_rows_kernel(u64 *out, const u64 *x, u64 c0, u64 c1, u32 lo, u32 hi, u32 logn,
                                       const u64 *cst, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)(hi - lo) * N;
    if (idx >= total) return;
    u32 t = lo + (u32)(idx >> logn);
    u32 n = (u32)(idx & (N - 1));
    size_t o = (size_t)t * N + n;
    u64 q = pd[t].q;
    out[o] = add_mod(out[o], mul_shoup(x[o], cst[2 * t], cst[2 * t + 1], q), q);
}

// a[r][n] *= 2^64 mod q, q the prime of row r (rows r % period: 0..period-1 = every prime of the chain)
__global__ void to_montgomery_kernel(u64 *a, u32 rows, u32 period, u32 logn, const PrimeDev *pd) {
    const u32 N = 1u << logn;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * N) return;
    const PrimeDev &P = pd[(u32)(idx >> logn) % period];
    a[idx] = mul_shoup(a[idx], P.r64, P.r64s, P.q);
}

static void make_ksk(Ctx *c, u64 *key, const u64 *sp, u32 key_id) {
    const u32 E = c->nprimes(), N = c->N;
    // [P]_{q_t} (Shoup pairs) for t < L1
    std::vector<u64> pm(2 * E, 0);
    for (u32 t = 0; t < c->L1; ++t) {
        u64 q = c->primes[t], v = 1;
        for (u32 k = 0; k < c->K; ++k) v = mulm(v, c->primes[c->L1 + k] % q, q);
        pm[2 * t] = v;
        pm[2 * t + 1] = (u64)(((unsigned __int128)v << 64) / q);
    }
    const u64 *pmd = c->const_table("Pmod", pm);
    DBuf e(c, (size_t)E * N), as(c, (size_t)E * N);
    for (u32 j = 0; j < c->dnum; ++j) {
        u64 *b = key + (size_t)j * 2 * E * N;
        u64 *a = b + (size_t)E * N;
        SeedList sl;
        sl.seed[0] = c->seed;
        sl.stream[0] = stream_id(RS_KSK_A, key_id, j, 0);
        sample_uniform(c, a, sl, 1, E, E, E, 0);
        ntt_forward(c, a, rows_regular(E, E, E, 0));
        sl.stream[0] = stream_id(RS_KSK_E, key_id, j, 0);
        sample_small(c, e.p, sl, 1, E, E, E, 0, 1);
        ntt_forward(c, e.p, rows_regular(E, E, E, 0));
        ew_binop(c, OP_MUL, as.p, a, c->sk.p, E, E, E, 0);
        ew_binop(c, OP_SUB, b, e.p, as.p, E, E, E, 0);
        u32 lo = j * c->alpha, hi = std::min(lo + c->alpha, c->L1);
        if (lo < hi) {
            size_t total = (size_t)(hi - lo) * N;
            prof_begin(c);
            add_scaled_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(b, sp, 0, 0, lo, hi,
                                                                                          c->logn, pmd, c->pdev);
            note_launch(c, "ksk_gadget");
        }
    }
    // stored in Montgomery form (times 2^64 mod q): the key-switch inner products
    // reduce their 128-bit sums with one Montgomery reduction
    const size_t total = (size_t)c->dnum * 2 * E * N;
    prof_begin(c);
    to_montgomery_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(key, c->dnum * 2 * E, E, c->logn,
                                                                              c->pdev);
    note_launch(c, "ksk_montgomery");
}

void keygen(Ctx *c, const std::vector<int> &steps) {
    const u32 E = c->nprimes(), N = c->N, L1 = c->L1;
    c->sk = DBuf(c, (size_t)E * N);
    SeedList sl;
    sl.seed[0] = c->seed;
    sl.stream[0] = stream_id(RS_SK, 0, 0, 0);
    sample_small(c, c->sk.p, sl, 1, E, E, E, 0, 0);
    ntt_forward(c, c->sk.p, rows_regular(E, E, E, 0));
    // public key (data primes)
    c->pk = DBuf(c, (size_t)2 * L1 * N);
    u64 *pk0 = c->pk.p, *pk1 = c->pk.p + (size_t)L1 * N;
    sl.stream[0] = stream_id(RS_PK_A, 0, 0, 0);
    sample_uniform(c, pk1, sl, 1, L1, L1, L1, 0);
    ntt_forward(c, pk1, rows_regular(L1, L1, L1, 0));
    DBuf e(c, (size_t)L1 * N), as(c, (size_t)L1 * N);
    sl.stream[0] = stream_id(RS_PK_E, 0, 0, 0);
    sample_small(c, e.p, sl, 1, L1, L1, L1, 0, 1);
    ntt_forward(c, e.p, rows_regular(L1, L1, L1, 0));
    ew_binop(c, OP_MUL, as.p, pk1, c->sk.p, L1, L1, L1, 0);
    ew_binop(c, OP_SUB, pk0, e.p, as.p, L1, L1, L1, 0);
    // relinearisation key: s' = s^2
    DBuf s2(c, (size_t)E * N);
    ew_binop(c, OP_MUL, s2.p, c->sk.p, c->sk.p, E, E, E, 0);
    c->rlk = DBuf(c, (size_t)c->dnum * 2 * E * N);
    make_ksk(c, c->rlk.p, s2.p, 0);
    // Galois keys: s' = sigma_g(s)
    c->gk.clear();
    c->gkp.clear();
    DBuf sg(c, (size_t)E * N);
    for (int st : steps) {
        u32 g = c->galois_elt(st);
        if (g == 1 || c->gk.count(g)) continue;
        galois_permute(c, sg.p, c->sk.p, E, g);
        DBuf k(c, (size_t)c->dnum * 2 * E * N);
        make_ksk(c, k.p, sg.p, g);
        // the same key with every limb permuted by sigma_g^{-1} (read coalesced by hoisted rotations)
        DBuf kp(c, (size_t)c->dnum * 2 * E * N);
        galois_permute(c, kp.p, k.p, c->dnum * 2 * E, c->galois_inverse(g));
        c->gk.emplace(g, std::move(k));
        c->gkp.emplace(g, std::move(kp));
    }
    c->have_keys = true;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
}

void require_key(Ctx *c, int step) {
    u32 g = c->galois_elt(step);
    if (g != 1 && !c->gk.count(g)) throw HeError(HE_ENOKEY, fmt("no Galois key for rotation step %d", step));
}

// ------------------------------------------------------------------ ciphertexts
size_t cts_ct_words(const Ctx *c, u32 lp) { return (size_t)2 * lp * c->N; }

Cts cts_alloc(Ctx *c, u32 B, u32 lp, double scale, const Layout &lay) {
    Cts t;
    t.mem = std::make_shared<DBuf>(c, (size_t)B * 2 * lp * c->N);
    t.off = 0;
    t.B = B;
    t.lp = lp;
    t.scale = scale;
    t.lay = lay;
    return t;
}

Cts cts_view(const Cts &base, size_t off_words, u32 B) {
    Cts t = base;
    t.off = base.off + off_words;
    t.B = B;
    return t;
}

Cts encrypt(Ctx *c, const double *x_dev, u32 W, u32 H, u32 nsamp, u32 spc, u32 stride, u64 enc_seed, u32 C) {
    if (!c->have_keys) throw HeError(HE_EINVAL, "he_keygen has not run");
    if (!nsamp || !C) throw HeError(HE_EINVAL, "no samples to encrypt");
    const u32 N = c->N, M = N / 2, L1 = c->L1;
    if (!spc || !stride || (u64)spc * stride > M || (u64)C * W * H > stride)
        throw HeError(HE_ESLOTS, "samples do not fit in the slots");
    const u32 B = (nsamp + spc - 1) / spc;
    Layout lay;
    lay.W_img = lay.W = W;
    lay.H_img = lay.H = H;
    lay.I = 1;
    lay.stride = stride;
    lay.n_samples = spc;
    lay.dims = H == 1 ? 1 : 2;
    lay.C = C;
    Cts out = cts_alloc(c, B, L1, c->scale, lay);
    DBuf z(c, (size_t)B * M);
    pack_samples(c, reinterpret_cast<double *>(z.p), x_dev, nsamp, spc, stride, C * W * H, B);
    for (u32 b0 = 0; b0 < B; b0 += SEEDLIST_MAX) {
        const u32 nb = std::min<u32>(SEEDLIST_MAX, B - b0);
        DBuf me(c, (size_t)nb * L1 * N), e1(c, (size_t)nb * L1 * N), u(c, (size_t)nb * L1 * N);
        encode_dense(c, me.p, reinterpret_cast<const double *>(z.p) + (size_t)b0 * M, nb, c->scale, L1, false);
        // encode_dense leaves evaluation form; the error is added in evaluation form as well
        SeedList sl;
        for (u32 i = 0; i < nb; ++i) sl.seed[i] = enc_seed + b0 + i;
        for (u32 i = 0; i < nb; ++i) sl.stream[i] = stream_id(RS_ENC_E0, 0, 0, 0);
        sample_small(c, e1.p, sl, nb, L1, L1, L1, 0, 1);
        ntt_forward(c, e1.p, rows_regular(nb * L1, L1, L1, 0));
        ew_binop(c, OP_ADD, me.p, me.p, e1.p, nb * L1, L1, L1, 0);
        for (u32 i = 0; i < nb; ++i) sl.stream[i] = stream_id(RS_ENC_E1, 0, 0, 0);
        sample_small(c, e1.p, sl, nb, L1, L1, L1, 0, 1);
        ntt_forward(c, e1.p, rows_regular(nb * L1, L1, L1, 0));
        for (u32 i = 0; i < nb; ++i) sl.stream[i] = stream_id(RS_ENC_U, 0, 0, 0);
        sample_small(c, u.p, sl, nb, L1, L1, L1, 0, 0);
        ntt_forward(c, u.p, rows_regular(nb * L1, L1, L1, 0));
        enc_combine(c, out.data() + (size_t)b0 * 2 * L1 * N, u.p, me.p, e1.p, L1, nb);
    }
    check_encode_errors(c);
    return out;
}

// ------------------------------------------------------------------ ops
static void same_shape(const Cts &a, const Cts &b) {
    if (a.B != b.B || a.lp != b.lp) throw HeError(HE_EINVAL, "ciphertext batch / level mismatch");
    if (a.scale != b.scale) throw HeError(HE_ESCALE, fmt("scale mismatch %.17g vs %.17g", a.scale, b.scale));
}

Cts ct_add(Ctx *c, const Cts &a, const Cts &b) {
    same_shape(a, b);
    Cts o = cts_alloc(c, a.B, a.lp, a.scale, a.lay);
    ew_binop(c, OP_ADD, o.data(), a.data(), b.data(), a.B * 2 * a.lp, a.lp, a.lp, 0);
    return o;
}

void ct_add_inplace(Ctx *c, Cts &a, const Cts &b) {
    same_shape(a, b);
    ew_binop(c, OP_ADD, a.data(), a.data(), b.data(), a.B * 2 * a.lp, a.lp, a.lp, 0);
}

Cts ct_rescale(Ctx *c, const Cts &a) {
    if (a.lp < 2) throw HeError(HE_ELEVEL, "rescale: no level left");
    Cts o = cts_alloc(c, a.B, a.lp - 1, a.scale / (double)c->primes[a.lp - 1], a.lay);
    rescale_batch(c, o.data(), a.data(), a.B, a.lp);
    return o;
}

// Drop-Level (Sec. IV-A) as a modulus drop: the top limbs of every polynomial are
// discarded down to `keep` limbs (exact; message and scale unchanged)
Cts ct_drop_to(Ctx *c, const Cts &a, u32 keep) {
    if (keep < 1 || keep > a.lp) throw HeError(HE_ELEVEL, "drop level: not that many levels left");
    if (keep == a.lp) return a;
    Cts o = cts_alloc(c, a.B, keep, a.scale, a.lay);
    CUDA_TRY(cudaMemcpy2DAsync(o.data(), (size_t)keep * c->N * 8, a.data(), (size_t)a.lp * c->N * 8,
                               (size_t)keep * c->N * 8, (size_t)a.B * 2, cudaMemcpyDeviceToDevice, c->stream));
    return o;
}

Cts ct_drop_level(Ctx *c, const Cts &a) {
    if (a.lp < 2) throw HeError(HE_ELEVEL, "drop level: no level left");
    return ct_drop_to(c, a, a.lp - 1);
}

Cts ct_mul_pt(Ctx *c, const Cts &a, const u64 *pt, double pt_scale) {
    Cts o = cts_alloc(c, a.B, a.lp, a.scale * pt_scale, a.lay);
    ew_bcast(c, OP_MUL, o.data(), a.data(), pt, a.B, a.lp, 3);
    return o;
}

void ct_add_pt_inplace(Ctx *c, Cts &a, const u64 *pt) { ew_bcast(c, OP_ADD, a.data(), a.data(), pt, a.B, a.lp, 1); }

static size_t acc_chunk(Ctx *c, u32 B, u32 lp, size_t nsteps) {
    const size_t per = (size_t)B * 2 * (lp + c->K) * c->N * 8;
    size_t lim = ((size_t)4 << 30) / (per ? per : 1);
    if (lim < 1) lim = 1;
    if (lim > KEYLIST_MAX) lim = KEYLIST_MAX;
    return std::min(lim, nsteps);
}

Cts ct_rotate_naf(Ctx *c, const Cts &a, int step, std::map<int64_t, Cts> *cache);

void ct_rotate_hoisted_into(Ctx *c, const Cts &a, const std::vector<int> &steps, u64 *out) {
    const u32 N = c->N, lp = a.lp, B = a.B, E = lp + c->K;
    const size_t ctw = (size_t)B * 2 * lp * N;
    if (c->naf) {   // power-of-two keys: chains sharing their prefixes
        std::map<int64_t, Cts> cache;
        for (size_t i = 0; i < steps.size(); ++i) {
            Cts r = ct_rotate_naf(c, a, steps[i], &cache);
            CUDA_TRY(cudaMemcpyAsync(out + i * ctw, r.data(), ctw * 8, cudaMemcpyDeviceToDevice, c->stream));
        }
        return;
    }
    std::vector<int> ks;      // positions that need a key switch
    for (size_t i = 0; i < steps.size(); ++i) {
        u32 g = c->galois_elt(steps[i]);
        if (g == 1)
            CUDA_TRY(cudaMemcpyAsync(out + i * ctw, a.data(), ctw * 8, cudaMemcpyDeviceToDevice, c->stream));
        else {
            require_key(c, steps[i]);
            ks.push_back((int)i);
        }
    }
    if (ks.empty()) return;
    DBuf D(c, (size_t)B * ks_digits(c, lp) * E * N);
    ks_modup(c, D.p, a.data() + (size_t)lp * N, (size_t)2 * lp * N, B, lp);
    size_t chunk = acc_chunk(c, B, lp, ks.size());
    DBuf acc(c, chunk * B * 2 * E * N);
    // consecutive output positions are written by one moddown launch when possible
    for (size_t s0 = 0; s0 < ks.size();) {
        size_t s1 = s0 + 1;
        while (s1 < ks.size() && s1 - s0 < chunk && ks[s1] == ks[s1 - 1] + 1) ++s1;
        KeyList kl;
        for (size_t s = s0; s < s1; ++s) {
            u32 g = c->galois_elt(steps[ks[s]]);
            kl.key[s - s0] = c->gk.at(g).p;
            kl.g[s - s0] = g;
        }
        u32 S = (u32)(s1 - s0);
        ks_inner(c, acc.p, D.p, kl, S, B, lp);
        ks_moddown(c, out + (size_t)ks[s0] * ctw, acc.p, a.data(), (size_t)2 * lp * N, 1, kl, S, B, lp);
        s0 = s1;
    }
}

std::vector<Cts> ct_rotate_hoisted(Ctx *c, const Cts &a, const std::vector<int> &steps) {
    Cts all = cts_alloc(c, a.B * (u32)steps.size(), a.lp, a.scale, a.lay);
    ct_rotate_hoisted_into(c, a, steps, all.data());
    std::vector<Cts> out;
    for (size_t i = 0; i < steps.size(); ++i) {
        Cts v = cts_view(all, i * (size_t)a.B * 2 * a.lp * c->N, a.B);
        out.push_back(v);
    }
    return out;
}

// The rotation step r (taken mod N/2, in (-N/4, N/4]) as the signed powers of two of its
// non-adjacent form (Reitwiesner 1960), lowest first.
std::vector<int> naf_terms(int64_t r, u32 slots) {
    int64_t v = ((r % (int64_t)slots) + slots) % slots;
    if (v > (int64_t)slots / 2) v -= slots;
    std::vector<int> out;
    for (int i = 0; v != 0; ++i) {
        if (v & 1) {
            const int64_t d = 2 - (((v % 4) + 4) % 4);   // v = 1 (mod 4) -> +1, 3 (mod 4) -> -1
            v -= d;
            out.push_back((int)(d * ((int64_t)1 << i)));
        }
        v /= 2;   // exact: v is even here
    }
    return out;
}

static Cts ct_rotate_direct(Ctx *c, const Cts &a, int step);

// Rot(a, r) with power-of-two keys: the rotations of naf_terms(r) one after another. cache
// (partial sum -> ciphertext) lets the rotations of one input share their common prefixes.
Cts ct_rotate_naf(Ctx *c, const Cts &a, int step, std::map<int64_t, Cts> *cache) {
    const std::vector<int> terms = naf_terms(step, c->N / 2);
    if (terms.empty()) return ct_rotate_direct(c, a, 0);   // a copy
    Cts cur = a;
    int64_t acc = 0;
    for (int t : terms) {
        acc += t;
        if (cache) {
            auto it = cache->find(acc);
            if (it != cache->end()) {
                cur = it->second;
                continue;
            }
        }
        cur = ct_rotate_direct(c, cur, t);
        if (cache) cache->emplace(acc, cur);
    }
    return cur;
}

Cts ct_rotate(Ctx *c, const Cts &a, int step) {
    return c->naf ? ct_rotate_naf(c, a, step, nullptr) : ct_rotate_direct(c, a, step);
}

// one rotation of a rotate-then-multiply combination: with power-of-two keys the chain of its
// non-adjacent form (cache: prefixes shared between the rotations of one input), else the
// step's own key switch (paper-order schedule)
static Cts rotate_seq(Ctx *c, const Cts &a, int step, std::map<int64_t, Cts> *cache) {
    return c->naf ? ct_rotate_naf(c, a, step, cache) : ct_rotate_direct(c, a, step);
}

static Cts ct_rotate_direct(Ctx *c, const Cts &a, int step) {
    const u32 N = c->N, lp = a.lp, B = a.B, E = lp + c->K;
    u32 g = c->galois_elt(step);
    Cts o = cts_alloc(c, B, lp, a.scale, a.lay);
    if (g == 1) {
        CUDA_TRY(cudaMemcpyAsync(o.data(), a.data(), (size_t)B * 2 * lp * N * 8, cudaMemcpyDeviceToDevice,
                                 c->stream));
        return o;
    }
    require_key(c, step);
    DBuf t(c, (size_t)B * 2 * lp * N);
    galois_permute(c, t.p, a.data(), B * 2 * lp, g);
    DBuf D(c, (size_t)B * ks_digits(c, lp) * E * N);
    ks_modup(c, D.p, t.p + (size_t)lp * N, (size_t)2 * lp * N, B, lp);
    KeyList kl;
    kl.key[0] = c->gk.at(g).p;
    kl.g[0] = 1;
    DBuf acc(c, (size_t)B * 2 * E * N);
    ks_inner(c, acc.p, D.p, kl, 1, B, lp);
    ks_moddown(c, o.data(), acc.p, t.p, (size_t)2 * lp * N, 1, kl, 1, B, lp);
    return o;
}

Cts ct_square(Ctx *c, const Cts &a) {
    const u32 N = c->N, lp = a.lp, B = a.B, E = lp + c->K;
    if (lp < 2) throw HeError(HE_ELEVEL, "square: no level left");
    DBuf d(c, (size_t)B * 3 * lp * N);
    tensor_square(c, d.p, a.data(), B, lp);
    DBuf D(c, (size_t)B * ks_digits(c, lp) * E * N);
    ks_modup(c, D.p, d.p + (size_t)2 * lp * N, (size_t)3 * lp * N, B, lp);
    KeyList kl;
    kl.key[0] = c->rlk.p;
    kl.g[0] = 1;
    DBuf acc(c, (size_t)B * 2 * E * N);
    if (c->literal) {
        // one step at a time: relinearise (ModDown of both accumulators, plus d0 / d1), then the
        // centred rescale
        ks_inner(c, acc.p, D.p, kl, 1, B, lp);
        Cts rl = cts_alloc(c, B, lp, a.scale * a.scale, a.lay);
        ks_moddown(c, rl.data(), acc.p, d.p, (size_t)3 * lp * N, 3, kl, 1, B, lp);
        return ct_rescale(c, rl);
    }
    // relinearise and rescale as one division by q_top * P: P * (d0, d1) joins the accumulators
    // in the inner product's own pass
    ks_inner(c, acc.p, D.p, kl, 1, B, lp, d.p, (size_t)3 * lp * N);
    Cts r = cts_alloc(c, B, lp - 1, a.scale * a.scale / (double)c->primes[lp - 1], a.lay);
    ks_moddown_rescale(c, r.data(), acc.p, B, lp);
    return r;
}

// Y = sum_i Rot(X_i, steps[i]) over the CH channels of X (CH*B ciphertexts, channel-major),
// with one ModDown: each channel's accumulator pair for its own step is summed over Q_l u P.
Cts ct_lincomb_diag(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<int> &steps) {
    const u32 N = c->N, lp = X.lp, E = lp + c->K, Bt = CH * B;
    if (X.B != Bt || steps.size() != CH) throw HeError(HE_EINVAL, "lincomb_diag: shape mismatch");
    if (seq_lincomb(c)) {   // each channel rotated on its own (a chain with power-of-two keys), then summed
        const size_t bw = (size_t)B * cts_ct_words(c, lp);
        Cts R = cts_alloc(c, Bt, lp, X.scale, X.lay);
        for (u32 i = 0; i < CH; ++i) {
            Cts r = rotate_seq(c, cts_view(X, i * bw, B), steps[i], nullptr);
            CUDA_TRY(cudaMemcpyAsync(R.data() + i * bw, r.data(), bw * 8, cudaMemcpyDeviceToDevice, c->stream));
        }
        Cts out = cts_alloc(c, B, lp, X.scale, X.lay);
        sum_stack(c, out.data(), R.data(), bw, CH, B * 2 * lp, lp, lp, c->L1, 0);
        return out;
    }
    const u32 beta = ks_digits(c, lp);
    bool any_ks = false;
    for (int s : steps)
        if (c->galois_elt(s) != 1) {
            require_key(c, s);
            any_ks = true;
        }
    DBuf D;
    if (any_ks) {
        D = DBuf(c, (size_t)Bt * beta * E * N);
        ks_modup(c, D.p, X.data() + (size_t)lp * N, (size_t)2 * lp * N, Bt, lp);
    }
    const size_t zw = (size_t)B * 2 * E * N;
    DBuf acc(c, (size_t)CH * zw);
    for (u32 i = 0; i < CH; ++i) {
        KeyList kl;
        const u32 g = c->galois_elt(steps[i]);
        kl.g[0] = g;
        kl.ginv[0] = c->galois_inverse(g);
        kl.key[0] = g == 1 ? nullptr : c->gk.at(g).p;
        kl.keyp[0] = g == 1 ? nullptr : c->gkp.at(g).p;
        const u64 *Di = any_ks ? D.p + (size_t)i * B * beta * E * N : nullptr;
        ks_lazy(c, acc.p + (size_t)i * zw, Di, X.data() + (size_t)i * B * cts_ct_words(c, lp), kl, 1, B, lp);
    }
    DBuf Z(c, zw);
    sum_stack(c, Z.p, acc.p, zw, CH, B * 2 * E, E, lp, c->L1, 0);
    Cts out = cts_alloc(c, B, lp, X.scale, X.lay);
    KeyList none;
    none.g[0] = 1;
    none.key[0] = nullptr;
    ks_moddown(c, out.data(), Z.p, nullptr, 0, 0, none, 1, B, lp);
    return out;
}

// Hoisted linear combination of rotations with one ModDown per output:
//   Y_o = sum_i sum_s w[o][i][s] (.) Rot(X_i, steps[s])
// X holds CH*B ciphertexts (channel-major).  pts: [O][S*CH][lp+K][N] plaintexts over
// Q_l u P with t = s*CH + i, or nullptr for the plain sums Y_i = sum_s Rot(X_i, steps[s])
// (one output per channel).  The weighted key-switch accumulators, with P*sigma(c0)
// folded in, are summed over Q_l u P and ModDown runs once per output ciphertext.
// One output from channels that each have their own steps (every channel the same count K):
//   Y = sum_i sum_k pts[i][k] (.) Rot(X_i, steps[i][k])
// X holds CH*B ciphertexts (channel-major); pts [CH][K][lp+K_sp][N] over Q_l u P (over Q_l
// with power-of-two keys).  Each channel's rotations share one ModUp; the weighted
// accumulators of every channel are summed over Q_l u P and ModDown (with rescale: the one
// division by q_top * P) runs once.
Cts ct_rotate_naf(Ctx *c, const Cts &a, int step, std::map<int64_t, Cts> *cache);

Cts ct_lincomb_chan(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<std::vector<int>> &steps, const u64 *pts,
                    double pt_scale, bool rescale) {
    const u32 N = c->N, lp = X.lp, Bt = CH * B;
    if (X.B != Bt || steps.size() != CH || !CH) throw HeError(HE_EINVAL, "lincomb_chan: shape mismatch");
    const u32 K = (u32)steps[0].size();
    for (const auto &st : steps) {
        if (st.size() != K || !K) throw HeError(HE_EINVAL, "lincomb_chan: steps per channel differ");
        for (int s : st)
            if (c->naf) {
                for (int t : naf_terms(s, N / 2)) require_key(c, t);
            } else if (c->galois_elt(s) != 1) {
                require_key(c, s);
            }
    }
    const size_t bw = (size_t)B * cts_ct_words(c, lp);   // one channel's block of B ciphertexts
    if (seq_lincomb(c)) {
        const size_t pw = (size_t)lp * N;
        Cts Z = cts_alloc(c, B, lp, X.scale * pt_scale, X.lay);
        Cts R = cts_alloc(c, K * B, lp, X.scale, X.lay);
        for (u32 i = 0; i < CH; ++i) {
            std::map<int64_t, Cts> cache;
            const Cts Xi = cts_view(X, i * bw, B);
            for (u32 k = 0; k < K; ++k) {
                Cts r = rotate_seq(c, Xi, steps[i][k], &cache);
                CUDA_TRY(cudaMemcpyAsync(R.data() + k * bw, r.data(), bw * 8, cudaMemcpyDeviceToDevice, c->stream));
            }
            mac(c, Z.data(), bw, R.data(), bw, pts + (size_t)i * K * pw, 1, K, B, lp, lp, c->L1, i > 0,
                (size_t)CH * K * pw);
        }
        return rescale ? ct_rescale(c, Z) : Z;
    }
    const u32 E = lp + c->K, beta = ks_digits(c, lp);
    DBuf D(c, (size_t)Bt * beta * E * N);
    ks_modup(c, D.p, X.data() + (size_t)lp * N, (size_t)2 * lp * N, Bt, lp);
    const size_t zw = (size_t)B * 2 * E * N;
    DBuf Z(c, zw);
    const size_t chunk = KEYLIST_MAX;
    for (u32 i = 0; i < CH; ++i) {
        for (u32 s0 = 0; s0 < K; s0 += (u32)chunk) {
            const u32 Sc = std::min<u32>((u32)chunk, K - s0);
            KeyList kl;
            for (u32 s = 0; s < Sc; ++s) {
                const u32 g = c->galois_elt(steps[i][s0 + s]);
                kl.g[s] = g;
                kl.ginv[s] = c->galois_inverse(g);
                kl.key[s] = g == 1 ? nullptr : c->gk.at(g).p;
                kl.keyp[s] = g == 1 ? nullptr : c->gkp.at(g).p;
            }
            // Z += sum_{k in chunk} pts[i][k] (.) A_k(X_i), the accumulators summed in registers
            ks_comb(c, Z.p, D.p + (size_t)i * B * beta * E * N, X.data() + i * bw, kl, Sc, 1, B, lp,
                    pts + ((size_t)i * K + s0) * E * N, 1, (size_t)K * E * N, i > 0 || s0 > 0);
        }
    }
    if (rescale) {
        if (lp < 2) throw HeError(HE_ELEVEL, "rescale: no level left");
        Cts out = cts_alloc(c, B, lp - 1, X.scale * pt_scale / (double)c->primes[lp - 1], X.lay);
        ks_moddown_rescale(c, out.data(), Z.p, B, lp);
        return out;
    }
    Cts out = cts_alloc(c, B, lp, X.scale * pt_scale, X.lay);
    KeyList none;
    none.g[0] = 1;
    none.key[0] = nullptr;
    ks_moddown(c, out.data(), Z.p, nullptr, 0, 0, none, 1, B, lp);
    return out;
}

// Rotate-then-multiply (power-of-two keys, and the paper-order schedule: Alg. 1 / Alg. 2 as
// printed).  The whole batch X is rotated by every step (chains sharing their prefixes with
// power-of-two keys, one key switch per step otherwise), the plaintexts pts [O][S*CH][lp][N]
// (over Q_l) multiply the rotations and the products are summed (or the rotations are
// summed); then the centred rescale.
static Cts ct_lincomb_seq(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<int> &steps, const u64 *pts,
                          u32 O, double pt_scale, bool rescale) {
    const u32 N = c->N, lp = X.lp, Bt = CH * B, S = (u32)steps.size();
    const size_t bw = (size_t)B * cts_ct_words(c, lp);   // one block of B ciphertexts
    Cts R = cts_alloc(c, S * Bt, lp, X.scale, X.lay);    // [s][channel][b]
    std::map<int64_t, Cts> cache;
    for (u32 s = 0; s < S; ++s) {
        Cts r = rotate_seq(c, X, steps[s], &cache);
        CUDA_TRY(cudaMemcpyAsync(R.data() + (size_t)s * CH * bw, r.data(), (size_t)CH * bw * 8,
                                 cudaMemcpyDeviceToDevice, c->stream));
    }
    cache.clear();
    const u32 nout = pts ? O : CH;
    Cts Z = cts_alloc(c, nout * B, lp, X.scale * (pts ? pt_scale : 1.0), X.lay);
    if (pts)
        mac(c, Z.data(), bw, R.data(), bw, pts, O, S * CH, B, lp, lp, c->L1, 0, (size_t)S * CH * lp * N);
    else
        sum_stack(c, Z.data(), R.data(), (size_t)CH * bw, S, CH * B * 2 * lp, lp, lp, c->L1, 0);
    return rescale ? ct_rescale(c, Z) : Z;
}

Cts ct_lincomb(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<int> &steps, const u64 *pts, u32 O,
               double pt_scale, bool rescale) {
    const u32 N = c->N, lp = X.lp, E = lp + c->K, Bt = CH * B, S = (u32)steps.size();
    if (X.B != Bt) throw HeError(HE_EINVAL, "lincomb: batch mismatch");
    if (seq_lincomb(c)) return ct_lincomb_seq(c, X, CH, B, steps, pts, O, pt_scale, rescale);
    bool any_ks = false;
    for (int s : steps)
        if (c->galois_elt(s) != 1) {
            require_key(c, s);
            any_ks = true;
        }
    DBuf D;
    if (any_ks) {
        D = DBuf(c, (size_t)Bt * ks_digits(c, lp) * E * N);
        ks_modup(c, D.p, X.data() + (size_t)lp * N, (size_t)2 * lp * N, Bt, lp);
    }
    const u32 nout = pts ? O : CH;   // outputs, each a batch of B ciphertexts
    const size_t zw = (size_t)B * 2 * E * N;    // one output batch over Q u P
    DBuf Z(c, (size_t)nout * zw);
    // the one-pass combination for plain sums and single outputs (measured: with four outputs, the
    // first convolution, the per-step accumulators with their shared key loads are faster)
    const bool comb = (!pts || O == 1) && (size_t)(pts ? B : Bt) <= 4 * 65535;
    // steps per chunk: bounded by the key list and, when per-step accumulators are kept, by ~16 GB of
    // them (every chunk after the first re-reads and re-writes the output accumulators, so one chunk
    // for the second LeNet-1 convolution's 25 steps of 256 ciphertexts, 11.7 GB)
    const size_t per_step = (size_t)Bt * 2 * E * N * 8;
    size_t chunk = comb ? KEYLIST_MAX : ((size_t)16 << 30) / (per_step ? per_step : 1);
    chunk = std::max<size_t>(1, std::min<size_t>(chunk, KEYLIST_MAX));
    DBuf acc;
    if (!comb) acc = DBuf(c, std::min<size_t>(chunk, S) * Bt * 2 * E * N);
    for (u32 s0 = 0; s0 < S; s0 += (u32)chunk) {
        const u32 Sc = std::min<u32>((u32)chunk, S - s0);
        KeyList kl;
        for (u32 s = 0; s < Sc; ++s) {
            u32 g = c->galois_elt(steps[s0 + s]);
            kl.g[s] = g;
            kl.ginv[s] = c->galois_inverse(g);
            kl.key[s] = g == 1 ? nullptr : c->gk.at(g).p;
            kl.keyp[s] = g == 1 ? nullptr : c->gkp.at(g).p;
        }
        if (comb) {
            // few outputs (pooling, the flatten's stages, FC, a first convolution): every step's
            // accumulator summed in registers, one pass, no per-step accumulators in memory
            ks_comb(c, Z.p, D.p, X.data(), kl, Sc, CH, B, lp, pts ? pts + (size_t)s0 * CH * E * N : nullptr, O,
                    (size_t)S * CH * E * N, s0 > 0);
            continue;
        }
        ks_lazy(c, acc.p, D.p, X.data(), kl, Sc, Bt, lp);
        if (pts) {
            // Z_o += sum_{t in chunk} pts[o][t] (.) acc[t], t = s*CH + i, blocks of B ciphertexts
            mac(c, Z.p, zw, acc.p, zw, pts + (size_t)s0 * CH * E * N, O, Sc * CH, B, E, lp, c->L1, s0 > 0,
                (size_t)S * CH * E * N);
        } else {
            // Z_i += sum_s acc[s][i]
            sum_stack(c, Z.p, acc.p, (size_t)Bt * 2 * E * N, Sc, Bt * 2 * E, E, lp, c->L1, s0 > 0);
        }
    }
    const double scale = X.scale * (pts ? pt_scale : 1.0);
    if (rescale) {
        if (lp < 2) throw HeError(HE_ELEVEL, "rescale: no level left");
        Cts out = cts_alloc(c, nout * B, lp - 1, scale / (double)c->primes[lp - 1], X.lay);
        ks_moddown_rescale(c, out.data(), Z.p, nout * B, lp);
        return out;
    }
    Cts out = cts_alloc(c, nout * B, lp, scale, X.lay);
    KeyList none;
    none.g[0] = 1;
    none.key[0] = nullptr;
    ks_moddown(c, out.data(), Z.p, nullptr, 0, 0, none, 1, nout * B, lp);
    return out;
}
