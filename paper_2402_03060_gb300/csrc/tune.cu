// tune.cu -- autotuner of launch shapes for the batched path.
//
// Every knob changes how work is laid out over CTAs, never the arithmetic, so
// all choices give bit-identical ciphertexts:
//   * limb layout (NTT, fused ModDown, fused rescale): one CTA per limb, a
//     2-CTA cluster per limb (half the shared memory and threads per CTA, so
//     more CTAs resident per SM, at the cost of one stage through DSMEM), or
//     two launches -- the outer stages over columns, the inner ten over
//     independent 1024-coefficient blocks (many small CTAs per SM);
//   * MAC output group: how many output accumulators one launch keeps in
//     registers (fewer: more resident warps, but the inputs are re-read per group);
//   * hoisted key-switch accumulation: ciphertexts per thread (key reuse in
//     registers vs. registers per thread) and grid order (coefficient tiles
//     fastest vs. ciphertext groups fastest, i.e. key-slice reuse in L2);
//   * one-pass combination (ks_comb): ciphertexts per thread.
// Each knob is timed with CUDA events on scratch data shaped like the context's
// top level (16 to 64 ciphertexts), the fastest kept; results are cached in a JSON
// file keyed by device name and parameters so a later process skips the sweep.
#include <stdio.h>
#include <string.h>

#include <functional>
#include <sstream>

#include "ntt_block.cuh"
#include "ops.cuh"

static bool layout_ok(int logn, int v) {
    if (v == NTT_TWO_KERNEL) return ntt2_ok(logn);
    if (v == 1) return ntt_can_split(logn);
    return v == 0 && !ntt_min_split(logn);
}

static int layout_default(int logn) { return logn >= 14 && ntt2_ok(logn) ? NTT_TWO_KERNEL : ntt_min_split(logn); }

int ntt_layout(const Ctx *c, int knob) {
    const int v = c->tuned[knob];
    if (v >= 0 && layout_ok(c->logn, v)) return v;
    return layout_default(c->logn);
}

namespace {

const char *knob_name[TUNE_COUNT] = {"ntt_split", "moddown_split", "rescale_split", "mac_group", "lazy_bt",
                                     "lazy_order", "mac_bk", "mac_split", "comb_bt", "comb_fold", "mac_tc"};

float time_ms(Ctx *c, const std::function<void()> &f) {
    f();   // warm-up
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        CUDA_TRY(cudaEventRecord(e0, c->stream));
        for (int k = 0; k < 3; ++k) f();
        CUDA_TRY(cudaEventRecord(e1, c->stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms / 3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// times f for every candidate value of knob; keeps the fastest, but stays with the first
// candidate (the default shape) unless another one is at least 2 % faster, so that timing
// noise does not flip the choice from one process to the next
void sweep(Ctx *c, int knob, const std::vector<int> &cands, const std::function<void()> &f, std::ostringstream &rep) {
    int best = cands[0];
    float best_ms = 1e30f, first_ms = 0;
    rep << "\"" << knob_name[knob] << "\": {";
    for (size_t i = 0; i < cands.size(); ++i) {
        c->tuned[knob] = cands[i];
        const float ms = time_ms(c, f);
        if (i == 0) first_ms = ms;
        rep << (i ? ", " : "") << "\"" << cands[i] << "\": " << ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = cands[i];
        }
    }
    if (best_ms > 0.98f * first_ms) best = cands[0];
    rep << ", \"chosen\": " << best << "}";
    c->tuned[knob] = best;
}

std::string cache_key(const Ctx *c) {
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, c->device));
    std::string k = fmt("v3|%s|sm%d%d|logn%d|L%u|K%u|dnum%u", prop.name, prop.major, prop.minor, c->logn, c->L1, c->K,
                        c->dnum);
    for (char &ch : k)
        if (ch == '"' || ch == '\\') ch = '_';
    return k;
}

// the cache: one line per key, {"key": {"knob": value, ...}, ...}
std::map<std::string, std::string> read_cache(const char *path) {
    std::map<std::string, std::string> m;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return m;
    char line[4096];
    while (fgets(line, sizeof line, f)) {
        const char *q0 = strchr(line, '"');
        if (!q0) continue;
        const char *q1 = strchr(q0 + 1, '"');
        const char *b0 = q1 ? strchr(q1, '{') : nullptr;
        const char *b1 = b0 ? strchr(b0, '}') : nullptr;
        if (!b1) continue;
        m[std::string(q0 + 1, q1)] = std::string(b0, b1 + 1);
    }
    fclose(f);
    return m;
}

void write_cache(const char *path, const std::map<std::string, std::string> &m) {
    FILE *f = fopen(path, "w");
    if (!f) throw HeError(HE_EINVAL, std::string("cannot write the tuning cache ") + path);
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : m) fprintf(f, "  \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++i < m.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
}

bool parse_entry(Ctx *c, const std::string &obj) {
    int v[TUNE_COUNT];
    for (int k = 0; k < TUNE_COUNT; ++k) {
        const std::string key = std::string("\"") + knob_name[k] + "\":";
        size_t p = obj.find(key);
        if (p == std::string::npos || sscanf(obj.c_str() + p + key.size(), " %d", &v[k]) != 1) return false;
    }
    for (int k = 0; k < TUNE_COUNT; ++k) c->tuned[k] = v[k];
    return true;
}

std::string entry_of(const Ctx *c) {
    std::string s = "{";
    for (int k = 0; k < TUNE_COUNT; ++k) s += fmt("%s\"%s\": %d", k ? ", " : "", knob_name[k], c->tuned[k]);
    return s + "}";
}

void measure(Ctx *c, std::ostringstream &rep) {
    const u32 N = c->N, lp = c->L1, K = c->K, E = lp + K, B = 16;
    const u32 beta = ks_digits(c, lp);
    // limb layouts this N allows, the default first (kept unless another is 2 % faster)
    std::vector<int> splits;
    {
        const int dflt = layout_default(c->logn);
        splits.push_back(dflt);
        for (int v : {0, 1, NTT_TWO_KERNEL})
            if (v != dflt && layout_ok(c->logn, v)) splits.push_back(v);
    }
    rep << "{";
    {   // NTT of 2*lp limbs of 16 ciphertexts
        DBuf a(c, (size_t)B * 2 * lp * N);
        CUDA_TRY(cudaMemsetAsync(a.p, 0, a.words * 8, c->stream));
        RowSet rs = rows_regular(B * 2 * lp, lp, lp, 0);
        sweep(c, TUNE_NTT, splits, [&] { ntt_forward(c, a.p, rs); }, rep);
    }
    {   // ModDown of 16 ciphertexts' accumulators, and rescale of 16 ciphertexts
        DBuf acc(c, (size_t)B * 2 * E * N), out(c, (size_t)B * 2 * lp * N);
        CUDA_TRY(cudaMemsetAsync(acc.p, 0, acc.words * 8, c->stream));
        KeyList kl;
        memset(&kl, 0, sizeof kl);
        kl.g[0] = 1;
        kl.ginv[0] = 1;
        rep << ", ";
        sweep(c, TUNE_MODDOWN, splits, [&] { ks_moddown(c, out.p, acc.p, nullptr, 0, 0, kl, 1, B, lp); }, rep);
        if (lp >= 2) {
            rep << ", ";
            sweep(c, TUNE_RESCALE, splits, [&] { rescale_batch(c, acc.p, out.p, B, lp); }, rep);
        }
    }
    {   // MAC: 12 outputs of 8 terms over Q u P (a convolution's shape)
        const u32 O = 12, T = 8, Bm = 32;
        DBuf pt(c, (size_t)O * T * E * N), x(c, (size_t)T * Bm * 2 * E * N), out(c, (size_t)O * Bm * 2 * E * N);
        CUDA_TRY(cudaMemsetAsync(pt.p, 0, pt.words * 8, c->stream));
        CUDA_TRY(cudaMemsetAsync(x.p, 0, x.words * 8, c->stream));
        rep << ", ";
        auto run = [&] {
            mac(c, out.p, (size_t)Bm * 2 * E * N, x.p, (size_t)Bm * 2 * E * N, pt.p, O, T, Bm, E, lp, c->L1, 0, 0);
        };
        c->tuned[TUNE_MAC_BK] = 64;
        c->tuned[TUNE_MAC_SPLIT] = 1;
        sweep(c, TUNE_MAC_GROUP, {12, 8, 6, 4}, run, rep);
        rep << ", ";
        sweep(c, TUNE_MAC_SPLIT, {1, 2}, run, rep);
        rep << ", ";
        sweep(c, TUNE_MAC_BK, {64, 32, 16}, run, rep);
    }
    {   // the same outputs over 48 terms: tensor cores or integer units
        const u32 O = 12, T = 48, Bm = 32;
        DBuf pt(c, (size_t)O * T * E * N), x(c, (size_t)T * Bm * 2 * E * N), out(c, (size_t)O * Bm * 2 * E * N);
        CUDA_TRY(cudaMemsetAsync(pt.p, 0, pt.words * 8, c->stream));
        CUDA_TRY(cudaMemsetAsync(x.p, 0, x.words * 8, c->stream));
        rep << ", ";
        sweep(c, TUNE_MAC_TC, {0, 5, 8}, [&] {
            mac(c, out.p, (size_t)Bm * 2 * E * N, x.p, (size_t)Bm * 2 * E * N, pt.p, O, T, Bm, E, lp, c->L1, 0, 0);
        }, rep);
    }
    if (beta <= 8) {   // hoisted key-switch accumulation: 16 steps of 64 ciphertexts (a convolution's shape)
        const u32 S = 16, B = 64;
        DBuf D(c, (size_t)B * beta * E * N), x(c, (size_t)B * 2 * lp * N), acc(c, (size_t)S * B * 2 * E * N);
        DBuf keys(c, (size_t)S * c->dnum * 2 * (c->L1 + K) * N);
        CUDA_TRY(cudaMemsetAsync(D.p, 0, D.words * 8, c->stream));
        CUDA_TRY(cudaMemsetAsync(x.p, 0, x.words * 8, c->stream));
        CUDA_TRY(cudaMemsetAsync(keys.p, 0, keys.words * 8, c->stream));
        KeyList kl;
        memset(&kl, 0, sizeof kl);
        for (u32 s = 0; s < S; ++s) {
            kl.g[s] = c->galois_elt((int64_t)s + 1);
            kl.ginv[s] = c->galois_inverse(kl.g[s]);
            kl.key[s] = kl.keyp[s] = keys.p + (size_t)s * c->dnum * 2 * (c->L1 + K) * N;
        }
        auto run = [&] { ks_lazy(c, acc.p, D.p, x.p, kl, S, B, lp); };
        const std::vector<int> bts = {2, 1, 4};
        rep << ", ";
        c->tuned[TUNE_LAZY_ORDER] = 0;
        sweep(c, TUNE_LAZY_BT, bts, run, rep);
        rep << ", ";
        sweep(c, TUNE_LAZY_ORDER, {0, 1}, run, rep);
        // the one-pass combination of a pooling's shape: three key-switched steps and the identity
        // summed per ciphertext
        KeyList kc = kl;
        kc.g[3] = 1;
        kc.key[3] = kc.keyp[3] = nullptr;
        DBuf z(c, (size_t)B * 2 * E * N);
        rep << ", ";
        sweep(c, TUNE_COMB_BT, {4, 2}, [&] { ks_comb(c, z.p, D.p, x.p, kc, 4, 1, B, lp, nullptr, 0, 0, 0); }, rep);
    }
    c->tuned[TUNE_COMB_FOLD] = COMB_FOLD_MIN_B;   // recorded, not timed
    rep << "}";
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->pool.release_cached();   // the scratch above goes back to the device
}

}  // namespace

const char *set_last_error(const char *msg);

extern "C" he_status he_autotune(he_ctx *h, const char *cache_path, char *report, size_t report_len) {
    try {
        if (!h || !h->c) throw HeError(HE_EINVAL, "null context");
        Ctx *c = h->c.get();
        CtxLock lk(c);
        CUDA_TRY(cudaSetDevice(c->device));
        const std::string key = cache_key(c);
        std::map<std::string, std::string> cache = read_cache(cache_path);
        std::string rep;
        auto it = cache.find(key);
        if (it != cache.end() && parse_entry(c, it->second)) {
            rep = "{\"cached\": " + it->second + "}";
        } else {
            const u64 launches = c->launches;
            const bool prof = c->profiling;
            c->profiling = false;
            std::ostringstream os;
            try {
                measure(c, os);
            } catch (...) {
                c->profiling = prof;
                c->launches = launches;
                throw;
            }
            c->profiling = prof;
            c->launches = launches;
            rep = os.str();
            if (cache_path) {
                cache[key] = entry_of(c);
                write_cache(cache_path, cache);
            }
        }
        if (report && report_len) {
            strncpy(report, rep.c_str(), report_len - 1);
            report[report_len - 1] = 0;
        }
        return HE_OK;
    } catch (const HeError &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HE_EINVAL;
    }
}

extern "C" he_status he_tuning_get(he_ctx *h, int32_t *values, size_t n) {
    if (!h || !h->c || !values) return HE_EINVAL;
    for (size_t k = 0; k < n && k < TUNE_COUNT; ++k) values[k] = h->c->tuned[k];
    return HE_OK;
}

extern "C" he_status he_tuning_set(he_ctx *h, const int32_t *values, size_t n) {
    if (!h || !h->c || !values) return HE_EINVAL;
    CtxLock lk(h->c.get());
    for (size_t k = 0; k < n && k < TUNE_COUNT; ++k) h->c->tuned[k] = values[k];
    return HE_OK;
}
