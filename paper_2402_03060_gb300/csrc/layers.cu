// layers.cu -- UniHENN's layers (paper Sec. IV), the layout planner (Sec. V),
// compiled models with batched / graph-replayed inference, and the C ABI.
//
// A feature map is held as ONE ciphertext batch of CH*B ciphertexts
// (channel-major: ciphertext index ch*B + b), so every per-channel operation
// of a layer -- rotations by the same steps, masks, squares, rescales -- is a
// single set of kernel launches over all channels and all ciphertexts.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <set>

#include "model.cuh"

// ------------------------------------------------------------------ helpers
struct Feat {
    Cts x;        // CH*B ciphertexts
    u32 CH = 1, B = 1;
    Cts chan(Ctx *c, u32 ch) const { return cts_view(x, (size_t)ch * B * cts_ct_words(c, x.lp), B); }
};

static std::vector<u32> valid_positions(const Layout &L, u32 Hout, u32 Wout, u32 Iout) {
    std::vector<u32> pos;
    for (u32 r = 0; r < Hout; ++r)
        for (u32 c = 0; c < Wout; ++c) pos.push_back(Iout * (r * L.W_img + c));
    return pos;
}

// encoded plaintexts for nv sparse slot vectors at level lp / scale; cached under key
static const u64 *get_pts(Ctx *c, PtCache *pc, const std::string &key, std::vector<DBuf> &tmp, const Layout &L,
                          const std::vector<u32> &off, const std::vector<u32> &pos, const std::vector<double> &val,
                          double scale, u32 lp, u32 ext = 0) {
    if (pc) {
        auto it = pc->pts.find(key);
        if (it != pc->pts.end()) return it->second.p;
    }
    u32 nv = (u32)off.size() - 1;
    Pool *saved = c->active;
    if (pc) c->active = nullptr;   // cached plaintexts live in the context pool
    DBuf out(c, (size_t)nv * (lp + ext) * c->N);
    c->active = saved;
    encode_sparse(c, out.p, key, off, pos, val, L.stride, L.n_samples, scale, lp, ext);
    u64 *p = out.p;
    if (pc)
        pc->pts.emplace(key, std::move(out));
    else
        tmp.push_back(std::move(out));
    return p;
}

// ------------------------------------------------------------------ layers
// Algorithm 1 (Sec. IV-B).  w: [co][ci][kh][kw].  Rotations Rot(C_in(i), I*(k + W_img*j));
// per output channel: sum of Mul(rot, K(o,i,j,k)) with K the weight (times the
// pending pooling factor) at every valid output slot, rescale, Add(bias at the
// valid output slots).  I_out = I*S.
static Feat layer_conv(Ctx *c, const Feat &in, const LayerSpec &sp, u32 kh, u32 kw, bool incremental, PtCache *pc,
                       const std::string &key) {
    const Layout &L = in.x.lay;
    const u32 ci = sp.ci, co = sp.co, S = sp.s, B = in.B, lp = in.x.lp, N = c->N;
    // an input of several channels in one ciphertext (Sec. III-A): input channel i is read
    // through the extra rotation i*W_img*H_img; all its rotations are hoisted together
    const bool packed = in.CH == 1 && L.prev == PREV_INPUT && L.C > 1;
    if (packed ? L.C != ci : in.CH != ci) throw HeError(HE_EINVAL, "conv: channel count mismatch");
    if (packed && incremental) throw HeError(HE_EINVAL, "conv: channels in one ciphertext need hoisted mode");
    if (lp < 2) throw HeError(HE_ELEVEL, "conv: no level left");
    if (kh > L.H || kw > L.W) throw HeError(HE_EINVAL, "conv: kernel larger than the feature map");
    const u32 Hout = (L.H - kh) / S + 1, Wout = (L.W - kw) / S + 1, Iout = L.I * S;
    const u32 KK = kh * kw;
    std::vector<int> steps;   // packed: step t = kk*ci + i, matching the plaintext order below
    for (u32 j = 0; j < kh; ++j)
        for (u32 k = 0; k < kw; ++k)
            for (u32 i = 0; i < (packed ? ci : 1u); ++i)
                steps.push_back((int)(i * L.W_img * L.H_img + L.I * (k + L.W_img * j)));
    const size_t ctw = cts_ct_words(c, lp);
    std::vector<u32> vpos = valid_positions(L, Hout, Wout, Iout);
    const u32 T = KK * ci;
    std::vector<DBuf> tmp;
    // plaintexts pt[o][off*ci + i]: the weight (times the pending factor) at every valid output slot
    auto weight_pts = [&](u32 ext) {
        std::vector<u32> off, pos;
        std::vector<double> val;
        const std::string k = key + (ext ? ":wx" : ":w");
        if (!pc || !pc->pts.count(k)) {
            off.push_back(0);
            for (u32 o = 0; o < co; ++o)
                for (u32 t = 0; t < T; ++t) {
                    u32 kk = t / ci, i = t % ci, j = kk / kw, k2 = kk % kw;
                    double wv = sp.w[(((size_t)o * ci + i) * kh + j) * kw + k2] * L.pending;
                    for (u32 p : vpos) {
                        pos.push_back(p);
                        val.push_back(wv);
                    }
                    off.push_back((u32)pos.size());
                }
        }
        return get_pts(c, pc, k, tmp, L, off, pos, val, c->scale, lp, ext);
    };
    Cts out;
    const u32 E2 = lp + ks_ext(c);
    const size_t per_out = (size_t)T * E2 * N;   // words of one output channel's masks
    if (!incremental && pc && pc->mask_budget && (size_t)co * per_out * 8 > pc->mask_budget) {
        // masks too large to keep: their sparse description is cached on the device and they
        // are encoded at every run, for groups of output channels that fit the budget
        const std::string dk = key + (ks_ext(c) ? ":wdx" : ":wd");
        if (!pc->pts.count(dk)) {
            std::vector<u32> off{0}, pos;
            std::vector<double> val;
            for (u32 o = 0; o < co; ++o)
                for (u32 t = 0; t < T; ++t) {
                    u32 kk = t / ci, i = t % ci, j = kk / kw, k2 = kk % kw;
                    double wv = sp.w[(((size_t)o * ci + i) * kh + j) * kw + k2] * L.pending;
                    for (u32 p : vpos) {
                        pos.push_back(p);
                        val.push_back(wv);
                    }
                    off.push_back((u32)pos.size());
                }
            const size_t o_pos = off.size() / 2 + 1, o_val = o_pos + pos.size() / 2 + 1;
            std::vector<u64> h(o_val + val.size(), 0);
            memcpy(h.data(), off.data(), off.size() * 4);
            memcpy(h.data() + o_pos, pos.data(), pos.size() * 4);
            memcpy(h.data() + o_val, val.data(), val.size() * 8);
            Pool *saved = c->active;
            c->active = nullptr;   // cached data lives in the context pool
            DBuf d(c, h.size());
            c->active = saved;
            CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));   // h is staged from the stack
            pc->pts.emplace(dk, std::move(d));
            pc->desc[dk] = {o_pos, o_val};
        }
        const u64 *d = pc->pts.at(dk).p;
        const std::vector<size_t> &dd = pc->desc.at(dk);
        const u32 *off_d = reinterpret_cast<const u32 *>(d);
        const u32 *pos_d = reinterpret_cast<const u32 *>(d + dd[0]);
        const double *val_d = reinterpret_cast<const double *>(d + dd[1]);
        const u32 og = (u32)std::max<size_t>(1, std::min<size_t>(co, pc->mask_budget / 8 / per_out));
        for (u32 o0 = 0; o0 < co; o0 += og) {
            const u32 oc = std::min(og, co - o0);
            DBuf m(c, (size_t)oc * per_out);
            for (u32 o = o0; o < o0 + oc; ++o)
                encode_sparse_dev(c, m.p + (size_t)(o - o0) * per_out, off_d + (size_t)o * T, T, pos_d, val_d,
                                  L.stride, L.n_samples, c->scale, lp, ks_ext(c));
            Cts r = ct_lincomb(c, in.x, packed ? 1 : ci, B, steps, m.p, oc, c->scale, true);
            if (o0 == 0) out = cts_alloc(c, co * B, r.lp, r.scale, r.lay);
            const size_t w = (size_t)oc * B * cts_ct_words(c, r.lp);
            CUDA_TRY(cudaMemcpyAsync(out.data() + (size_t)o0 * B * cts_ct_words(c, r.lp), r.data(), w * 8,
                                     cudaMemcpyDeviceToDevice, c->stream));
        }
    } else if (!incremental) {
        // one hoisted linear combination per output channel, ModDown and rescale as one division each
        const u64 *pts = weight_pts(ks_ext(c));
        out = ct_lincomb(c, in.x, packed ? 1 : ci, B, steps, pts, co, c->scale, true);
    } else {
        // rotated inputs R[off][ch*B + b]  (T index = off*ci + ch)
        Cts R = cts_alloc(c, KK * ci * B, lp, in.x.scale, L);
        CUDA_TRY(cudaMemcpyAsync(R.data(), in.x.data(), (size_t)ci * B * ctw * 8, cudaMemcpyDeviceToDevice,
                                 c->stream));
        for (u32 t = 1; t < KK; ++t) {
            u32 k = t % kw;
            int st = (int)(k > 0 ? L.I : L.I * (L.W_img - kw + 1));
            Cts prev = cts_view(R, (size_t)(t - 1) * ci * B * ctw, ci * B);
            Cts r = ct_rotate(c, prev, st);
            CUDA_TRY(cudaMemcpyAsync(R.data() + (size_t)t * ci * B * ctw, r.data(), (size_t)ci * B * ctw * 8,
                                     cudaMemcpyDeviceToDevice, c->stream));
        }
        const u64 *pts = weight_pts(0);
        Cts acc = cts_alloc(c, co * B, lp, in.x.scale * c->scale, L);
        // R[off][i*B + b] is block t = off*ci + i of B ciphertexts
        mac(c, acc.data(), (size_t)B * ctw, R.data(), (size_t)B * ctw, pts, co, T, B, lp);
        out = ct_rescale(c, acc);
    }
    {
        std::vector<u32> off, pos;
        std::vector<double> val;
        if (!pc || !pc->pts.count(key + ":b")) {
            off.push_back(0);
            for (u32 o = 0; o < co; ++o) {
                for (u32 p : vpos) {
                    pos.push_back(p);
                    val.push_back(sp.b[o]);
                }
                off.push_back((u32)pos.size());
            }
        }
        const u64 *bp = get_pts(c, pc, key + ":b", tmp, L, off, pos, val, out.scale, lp - 1);
        add_plain_multi(c, out.data(), bp, co, B, lp - 1, (size_t)B * cts_ct_words(c, lp - 1));
    }
    Layout L2 = L;
    L2.W = Wout;
    L2.H = Hout;
    L2.I = Iout;
    L2.pending = 1.0;
    L2.prev = PREV_CONV;
    L2.C = 1;
    out.lay = L2;
    Feat f;
    f.x = out;
    f.CH = co;
    f.B = B;
    (void)N;
    return f;
}

// Sec. IV-C: c x c average pooling by rotations and additions, no level; 1/c^2 deferred.
static Feat layer_avgpool(Ctx *c, const Feat &in, u32 cc) {
    const Layout &L = in.x.lay;
    const u32 ch = L.dims == 2 ? cc : 1;
    std::vector<int> steps;
    for (u32 j = 0; j < ch; ++j)
        for (u32 k = 0; k < cc; ++k) steps.push_back((int)(L.I * (k + L.W_img * j)));
    const u32 Bt = in.CH * in.B;
    Cts out = ct_lincomb(c, in.x, 1, Bt, steps, nullptr, 0, 1.0);
    Layout L2 = L;
    L2.W = L.W / cc;
    L2.H = L.dims == 2 ? L.H / cc : 1;
    L2.I = L.I * cc;
    L2.pending = L.pending / (double)(L.dims == 2 ? cc * cc : cc);
    L2.prev = PREV_POOL;
    out.lay = L2;
    Feat f = in;
    f.x = out;
    return f;
}

// square activation: Mul (C), relinearise, rescale; pending p -> p^2
static Feat layer_square(Ctx *c, const Feat &in) {
    Feat f = in;
    f.x = ct_square(c, in.x);
    f.x.lay.pending = in.x.lay.pending * in.x.lay.pending;
    return f;
}

// Approximate ReLU f(x) = c0 + c1 x + c2 x^2 (Sec. IV-F), 2 levels.  A pending pooling factor p
// is folded in: f(p x) = c0 + (c1 p) x + (c2 p^2) x^2 (Sec. IV-C).  a = Rescale(Mul(x^2, c2 p^2));
// b = Rescale(Mul(x, c1 p)) with the plaintext encoded at the scale that lands b on a's scale,
// then its top limb dropped to a's level; f = a + b + c0.  The constants sit at the valid slots
// only, so every other slot ends at zero.
static const double RELU_C0 = 0.375373, RELU_C1 = 0.5, RELU_C2 = 0.117071;

static Feat layer_approx_relu(Ctx *c, const Feat &in, PtCache *pc, const std::string &key) {
    const Layout &L = in.x.lay;
    const u32 lp = in.x.lp;
    if (lp < 3) throw HeError(HE_ELEVEL, "approximate ReLU: needs two levels");
    std::vector<u32> pos;
    if (L.prev == PREV_FLAT || L.prev == PREV_FC) {
        for (u32 t = 0; t < L.D; ++t) pos.push_back(t);
    } else {
        const u32 H = L.dims == 2 ? L.H : 1;
        for (u32 r = 0; r < H; ++r)
            for (u32 cc = 0; cc < L.W; ++cc) pos.push_back(L.I * (r * L.W_img + cc));
    }
    const double p = L.pending;
    std::vector<DBuf> tmp;
    auto mask = [&](const std::string &k, double v, double scale, u32 level) {
        std::vector<u32> off, ps;
        std::vector<double> val;
        if (!pc || !pc->pts.count(k)) {
            off = {0, (u32)pos.size()};
            ps = pos;
            val.assign(pos.size(), v);
        }
        return get_pts(c, pc, k, tmp, L, off, ps, val, scale, level);
    };
    Cts s2 = ct_square(c, in.x);                                              // level lp-1
    const u64 *m2 = mask(key + ":r2", RELU_C2 * p * p, c->scale, lp - 1);
    Cts a = ct_rescale(c, ct_mul_pt(c, s2, m2, c->scale));                    // level lp-2
    const double sb = a.scale * (double)c->primes[lp - 1] / in.x.scale;
    const u64 *m1 = mask(key + ":r1", RELU_C1 * p, sb, lp);
    Cts b = ct_drop_level(c, ct_rescale(c, ct_mul_pt(c, in.x, m1, sb)));       // level lp-2
    b.scale = a.scale;
    Cts y = ct_add(c, a, b);
    const u64 *m0 = mask(key + ":r0", RELU_C0, a.scale, lp - 2);
    ct_add_pt_inplace(c, y, m0);
    y.lay.pending = 1.0;
    Feat f = in;
    f.x = y;
    return f;
}

// The flatten's last masked stage (K steps) is merged with the packing of CH channels when the
// merged combination needs at most this many rotation steps (K*CH Galois keys instead of K + CH);
// never in the paper-order schedule
static const u32 MERGE_MAX_STEPS = 128;
static bool merge_last_stage(u32 k, u32 ch, bool literal) { return !literal && ch > 1 && k * ch <= MERGE_MAX_STEPS; }

// Sec. IV-E: remove intervals / invalid values, pack the channels.
// Every mask-rotate-sum stage  sum_k Rot(m_k (.) x, r_k)  is evaluated as one hoisted
// combination  sum_k Rot(m_k, r_k) (.) Rot(x, r_k)  (the masks are rotated in the clear),
// followed by one rescale.  The last stage and the channel packing (channel o rotated right
// by o*W*H) are one combination: channel o's terms use the steps r_k - o*W*H and the masks
// rotated by them, with one ModDown and rescale for the packed output.
// In the paper-order schedule a stage is the steps as listed: each mask multiplied with the
// ciphertext over Q_l, each product rotated left by its own key switch, the rotations added,
// then the centred rescale; the packing follows the last stage.
static Feat layer_flatten(Ctx *c, const Feat &in, PtCache *pc, const std::string &key) {
    const Layout &L = in.x.lay;
    const u32 I = L.I, W = L.W, H = L.H, Wi = L.W_img, CH = in.CH;
    const u32 M = c->N / 2;
    std::vector<DBuf> tmp;
    Cts cur = in.x;
    double pending = L.pending;
    struct Stage {
        std::string name;
        std::vector<std::vector<u32>> pos;   // within-sample positions of each mask
        std::vector<int> steps;
        double v;
    };
    std::vector<Stage> stages;
    // masks (within-sample positions, one value each) rotated left by their steps and
    // replicated over every sample position, encoded over Q_l u P at the input level;
    // mask j of the list uses pos[mk[j]] rotated by st[j]
    auto masks = [&](const std::string &name, const Stage &S, const std::vector<u32> &mk, const std::vector<int> &st,
                     u32 lp) {
        std::vector<u32> off, apos;
        std::vector<double> val;
        if (!pc || !pc->pts.count(name)) {
            off.push_back(0);
            for (size_t j = 0; j < mk.size(); ++j) {
                for (u32 b = 0; b < L.n_samples; ++b)
                    for (u32 p : S.pos[mk[j]]) {
                        int64_t a = ((int64_t)b * L.stride + p - st[j]) % (int64_t)M;
                        apos.push_back((u32)(a < 0 ? a + M : a));
                        val.push_back(S.v);
                    }
                off.push_back((u32)apos.size());
            }
        }
        Layout flat = L;
        flat.n_samples = 1;
        flat.stride = M;
        return get_pts(c, pc, name, tmp, flat, off, apos, val, c->scale, lp, ks_ext(c));
    };
    auto run_stage = [&](const Cts &x, const Stage &S) {
        std::vector<u32> mk;
        for (u32 k = 0; k < S.steps.size(); ++k) mk.push_back(k);
        if (c->literal) {
            const u32 K = (u32)S.steps.size(), B = x.B, lp = x.lp;
            const size_t bw = (size_t)B * cts_ct_words(c, lp);
            const u64 *pts = masks(key + S.name + ":lit", S, mk, std::vector<int>(K, 0), lp);   // not rotated
            Cts Y = cts_alloc(c, K * B, lp, x.scale * c->scale, x.lay);   // Y_k = m_k (.) x
            mac(c, Y.data(), bw, x.data(), bw, pts, K, 1, B, lp);
            Cts R = cts_alloc(c, K * B, lp, Y.scale, x.lay);
            for (u32 k = 0; k < K; ++k) {
                Cts r = ct_rotate(c, cts_view(Y, k * bw, B), S.steps[k]);
                CUDA_TRY(cudaMemcpyAsync(R.data() + k * bw, r.data(), bw * 8, cudaMemcpyDeviceToDevice, c->stream));
            }
            Cts Z = cts_alloc(c, B, lp, Y.scale, x.lay);
            sum_stack(c, Z.data(), R.data(), bw, K, B * 2 * lp, lp, lp, c->L1, 0);
            return ct_rescale(c, Z);
        }
        const u64 *pts = masks(key + S.name, S, mk, S.steps, x.lp);
        return ct_lincomb(c, x, 1, x.B, S.steps, pts, 1, c->scale, true);
    };
    if (L.prev == PREV_POOL) {
        Stage S{":cols", std::vector<std::vector<u32>>(W), {}, pending};
        for (u32 cc = 0; cc < W; ++cc) {
            for (u32 r = 0; r < H; ++r) S.pos[cc].push_back(I * (r * Wi + cc));
            S.steps.push_back((int)(cc * (I - 1)));
        }
        stages.push_back(S);
        pending = 1.0;
    } else if (L.prev == PREV_CONV) {
        if (pending != 1.0) throw HeError(HE_EINVAL, "flatten: unexpected pending factor");
        if (I > 1 && W > 1) {
            std::vector<int> st;
            for (u32 m = 0; m < I; ++m) st.push_back((int)(m * (I - 1)));
            cur = ct_lincomb(c, cur, 1, cur.B, st, nullptr, 0, 1.0);
            const u32 nblk = (W + I - 1) / I;
            Stage S{":blks", std::vector<std::vector<u32>>(nblk), {}, 1.0};
            for (u32 u = 0; u < nblk; ++u) {
                for (u32 r = 0; r < H; ++r)
                    for (u32 cc = I * u; cc < std::min(I * u + I, W); ++cc)
                        S.pos[u].push_back(I * r * Wi + I * I * u + (cc - I * u));
                S.steps.push_back((int)(u * I * (I - 1)));
            }
            stages.push_back(S);
        }
    } else {
        throw HeError(HE_EINVAL, "flatten must follow a convolution or an average pooling");
    }
    if (H > 1) {
        Stage S{":rows", std::vector<std::vector<u32>>(H), {}, 1.0};
        for (u32 r = 0; r < H; ++r) {
            for (u32 cc = 0; cc < W; ++cc) S.pos[r].push_back(I * r * Wi + cc);
            S.steps.push_back((int)(r * (Wi * I - W)));
        }
        stages.push_back(S);
    }
    for (size_t k = 0; k + 1 < stages.size(); ++k) cur = run_stage(cur, stages[k]);
    if (!stages.empty() && !merge_last_stage((u32)stages.back().steps.size(), CH, c->literal)) {
        cur = run_stage(cur, stages.back());
        stages.clear();
    }
    Cts acc;
    if (stages.empty()) {
        if (CH > 1) {   // pack: channel o rotated right by o*W*H, one ModDown for the sum
            std::vector<int> steps;
            for (u32 o = 0; o < CH; ++o) steps.push_back(-(int)(o * W * H));
            acc = ct_lincomb_diag(c, cur, CH, in.B, steps);
        } else {
            acc = cur;
        }
    } else if (CH == 1) {
        acc = run_stage(cur, stages.back());
    } else {
        const Stage &S = stages.back();
        std::vector<std::vector<int>> st(CH);
        std::vector<u32> mk;
        std::vector<int> flat_st;
        for (u32 o = 0; o < CH; ++o)
            for (u32 k = 0; k < S.steps.size(); ++k) {
                st[o].push_back(S.steps[k] - (int)(o * W * H));
                mk.push_back(k);
                flat_st.push_back(st[o].back());
            }
        const u64 *pts = masks(key + S.name + ":pack", S, mk, flat_st, cur.lp);
        acc = ct_lincomb_chan(c, cur, CH, in.B, st, pts, c->scale, true);
    }
    Layout L2 = L;
    L2.pending = pending;
    L2.prev = PREV_FLAT;
    L2.D = CH * W * H;
    L2.W = L2.D;
    L2.H = 1;
    L2.I = 1;
    acc.lay = L2;
    Feat f;
    f.CH = 1;
    f.B = in.B;
    f.x = acc;
    return f;
}

// Algorithm 2 (Sec. IV-D) on a flattened ciphertext; M [dout][din]
// sum_{i<m} Rot(x, i*d), the last step of Alg. 2: one hoisted combination of the m
// rotations (as printed), or (tree) binary doubling T_1 = x, T_2k = T_k + Rot(T_k, k*d)
// and the blocks T_{2^b} of the set bits of m, high to low, each rotated by the total
// of the blocks before it -- about log2(m) + popcount(m) rotations.
static Cts rotation_sum(Ctx *c, const Cts &x, u32 B, u32 d, u32 m, bool tree) {
    if (!tree || m == 1) {
        std::vector<int> st;
        for (u32 i = 0; i < m; ++i) st.push_back((int)(i * d));
        return ct_lincomb(c, x, 1, B, st, nullptr, 0, 1.0);
    }
    std::vector<Cts> T{x};   // T[b] = T_{2^b}
    for (u32 k = 1; 2 * k <= m; k *= 2) T.push_back(ct_add(c, T.back(), ct_rotate(c, T.back(), (int)(k * d))));
    Cts acc;
    bool have = false;
    u32 off = 0;
    for (int b = (int)T.size() - 1; b >= 0; --b) {
        if (!((m >> b) & 1)) continue;
        Cts term = off == 0 ? T[b] : ct_rotate(c, T[b], (int)(off * d));
        acc = have ? ct_add(c, acc, term) : term;
        have = true;
        off += 1u << b;
    }
    return acc;
}

static Feat layer_fc(Ctx *c, const Feat &in, const LayerSpec &sp, PtCache *pc, const std::string &key) {
    const Layout &L = in.x.lay;
    const u32 din = sp.ci, dout = sp.co, B = in.B;
    if (in.CH != 1 || (L.prev != PREV_FLAT && L.prev != PREV_FC)) throw HeError(HE_EINVAL, "FC needs a flattened input");
    if (din != L.D) throw HeError(HE_EINVAL, fmt("FC expects %u inputs, layout has %u", din, L.D));
    if (in.x.lp < 2) throw HeError(HE_ELEVEL, "FC: no level left");
    const u32 Wv = (din + dout - 1) / dout * dout;
    // steps: o for o < dout, then o - Wv for 1 <= o < dout
    std::vector<int> steps;
    for (u32 o = 0; o < dout; ++o) steps.push_back((int)o);
    for (u32 o = 1; o < dout; ++o) steps.push_back((int)o - (int)Wv);
    const u32 T = (u32)steps.size();
    const u32 lp = in.x.lp;
    const size_t ctw = cts_ct_words(c, lp);
    std::vector<DBuf> tmp;
    const u64 *pts;
    {
        std::vector<u32> off, pos;
        std::vector<double> val;
        if (!pc || !pc->pts.count(key + ":wx")) {
            // M_rot[o][t] = M_pad[t mod dout][(t + o) mod Wv] (times the pending factor)
            auto mrot = [&](u32 o, u32 t) -> double {
                u32 row = t % dout, col = (t + o) % Wv;
                if (col >= din) return 0.0;
                double m = sp.w[(size_t)row * din + col];
                return L.pending != 1.0 ? m * L.pending : m;
            };
            off.push_back(0);
            for (u32 o = 0; o < dout; ++o) {   // V1_o: t < Wv - o
                for (u32 t = 0; t < Wv - o; ++t) {
                    pos.push_back(t);
                    val.push_back(mrot(o, t));
                }
                off.push_back((u32)pos.size());
            }
            for (u32 o = 1; o < dout; ++o) {   // V2_o: t >= Wv - o
                for (u32 t = Wv - o; t < Wv; ++t) {
                    pos.push_back(t);
                    val.push_back(mrot(o, t));
                }
                off.push_back((u32)pos.size());
            }
        }
        pts = get_pts(c, pc, key + ":wx", tmp, L, off, pos, val, c->scale, lp, ks_ext(c));
    }
    (void)T;
    (void)ctw;
    // C_sum: every rotation of the input with its V1 / V2 vector, one ModDown
    Cts cs = ct_lincomb(c, in.x, 1, B, steps, pts, 1, c->scale, true);
    // C_out = sum_i Rot(C_sum, i * dout); FC field k = 1 selects the tree form
    Cts out = rotation_sum(c, cs, B, dout, Wv / dout, sp.k == 1);
    {
        std::vector<u32> off{0}, pos;
        std::vector<double> val;
        if (!pc || !pc->pts.count(key + ":b")) {
            for (u32 t = 0; t < dout; ++t) {
                pos.push_back(t);
                val.push_back(sp.b[t]);
            }
            off.push_back((u32)pos.size());
        }
        const u64 *bp = get_pts(c, pc, key + ":b", tmp, L, off, pos, val, out.scale, out.lp);
        ct_add_pt_inplace(c, out, bp);
    }
    Layout L2 = L;
    L2.pending = 1.0;
    L2.prev = PREV_FC;
    L2.D = dout;
    L2.W = dout;
    out.lay = L2;
    Feat f;
    f.x = out;
    f.CH = 1;
    f.B = B;
    return f;
}

// ------------------------------------------------------------------ planner
// Sec. V: the slots one sample needs = max(input W*H (Theorem 1 keeps every later
// valid value inside it), CH*W*H of a flatten, W_vec of an FC); levels and steps.
static Plan plan_layers(const std::vector<LayerSpec> &ls, u32 Wi, u32 Hi, bool literal) {
    const u32 dims = Hi == 1 ? 1 : 2;
    // the input's channels: CH_in of a first convolution, all in one ciphertext (Sec. III-A)
    const u32 C = !ls.empty() && (ls[0].op == HE_CONV2D || ls[0].op == HE_CONV1D) ? ls[0].ci : 1;
    if (C < 1 || (C > 1 && dims == 1)) throw HeError(HE_EINVAL, "input channels need a 2-D image");
    if ((u64)C * Wi * Hi > (1u << 30)) throw HeError(HE_EINVAL, "input too large");
    u32 W = Wi, H = Hi, I = 1, ch = 1, need = C * Wi * Hi, levels = 0;
    int prev = PREV_INPUT;
    std::set<int> st;
    for (const LayerSpec &s : ls) {
        if (s.op == HE_CONV2D || s.op == HE_CONV1D) {
            u32 kh = s.op == HE_CONV2D ? s.k : 1, kw = s.k;
            if (s.op == HE_CONV2D && dims == 1) throw HeError(HE_EINVAL, "conv2d on a 1-D input");
            if (kh > H || kw > W || s.s < 1) throw HeError(HE_EINVAL, "conv kernel does not fit");
            const u32 nch = prev == PREV_INPUT ? C : 1;
            for (u32 i = 0; i < nch; ++i)
                for (u32 j = 0; j < kh; ++j)
                    for (u32 k = 0; k < kw; ++k) st.insert((int)(i * Wi * Hi + I * (k + Wi * j)));
            H = (H - kh) / s.s + 1;
            W = (W - kw) / s.s + 1;
            I *= s.s;
            ch = s.co;
            levels += 1;
            prev = PREV_CONV;
        } else if (s.op == HE_SQUARE) {
            levels += 1;
        } else if (s.op == HE_APPROX_RELU) {
            levels += 2;
        } else if (s.op == HE_AVGPOOL) {
            u32 c = s.k, ckh = dims == 2 ? c : 1;
            if (c < 1 || c > W) throw HeError(HE_EINVAL, "pool size does not fit");
            for (u32 j = 0; j < ckh; ++j)
                for (u32 k = 0; k < c; ++k) st.insert((int)(I * (k + Wi * j)));
            W /= c;
            H = dims == 2 ? H / c : 1;
            I *= c;
            prev = PREV_POOL;
        } else if (s.op == HE_FLATTEN || s.op == HE_FC) {
            if (prev == PREV_CONV || prev == PREV_POOL) {
                std::vector<std::vector<int>> stage;   // steps of the masked stages, in order
                if (prev == PREV_POOL) {
                    levels += 1;
                    stage.emplace_back();
                    for (u32 c = 0; c < W; ++c) stage.back().push_back((int)(c * (I - 1)));
                } else if (I > 1 && W > 1) {
                    levels += 1;
                    for (u32 m = 0; m < I; ++m) st.insert((int)(m * (I - 1)));
                    stage.emplace_back();
                    for (u32 u = 0; u < (W + I - 1) / I; ++u) stage.back().push_back((int)(u * I * (I - 1)));
                }
                if (H > 1) {
                    levels += 1;
                    stage.emplace_back();
                    for (u32 r = 0; r < H; ++r) stage.back().push_back((int)(r * (Wi * I - W)));
                }
                if (!stage.empty() && merge_last_stage((u32)stage.back().size(), ch, literal)) {
                    // the last stage merged with the channel packing
                    for (size_t k = 0; k + 1 < stage.size(); ++k) st.insert(stage[k].begin(), stage[k].end());
                    for (int sk : stage.back())
                        for (u32 o = 0; o < ch; ++o) st.insert(sk - (int)(o * W * H));
                } else {
                    for (const auto &v : stage) st.insert(v.begin(), v.end());
                    for (u32 o = 0; o < ch; ++o) st.insert(-(int)(o * W * H));
                }
                need = std::max(need, ch * W * H);
                prev = PREV_FLAT;
                W = ch * W * H;
                H = 1;
                I = 1;
                ch = 1;
            }
            if (s.op == HE_FC) {
                if (prev != PREV_FLAT && prev != PREV_FC) throw HeError(HE_EINVAL, "FC needs a flattened input");
                if (s.ci != W) throw HeError(HE_EINVAL, fmt("FC DAT_in %u does not match %u", s.ci, W));
                u32 Wv = (s.ci + s.co - 1) / s.co * s.co;
                need = std::max(need, Wv);
                for (u32 o = 0; o < s.co; ++o) st.insert((int)o);
                for (u32 o = 1; o < s.co; ++o) st.insert((int)o - (int)Wv);
                const u32 m = Wv / s.co;
                if (s.k == 1) {   // tree form of the final rotation sum
                    u32 k = 1;
                    for (; 2 * k <= m; k *= 2) st.insert((int)(k * s.co));
                    u32 off = 0;
                    for (int b = 31; b >= 0; --b)
                        if ((m >> b) & 1) {
                            if (off) st.insert((int)(off * s.co));
                            off += 1u << b;
                        }
                } else {
                    for (u32 i = 0; i < m; ++i) st.insert((int)(i * s.co));
                }
                levels += 1;
                prev = PREV_FC;
                W = s.co;
            }
        } else {
            throw HeError(HE_EINVAL, "unknown layer op");
        }
    }
    st.erase(0);
    Plan p;
    p.stride = need;
    p.levels = levels;
    p.C = C;
    p.steps.assign(st.begin(), st.end());
    return p;
}

static std::vector<LayerSpec> copy_layers(const he_layer *layers, size_t n, u32 Hi) {
    std::vector<LayerSpec> out;
    for (size_t i = 0; i < n; ++i) {
        const he_layer &l = layers[i];
        LayerSpec s;
        s.op = l.op;
        s.ci = l.ch_in;
        s.co = l.ch_out;
        s.k = l.k;
        s.s = l.stride ? l.stride : 1;
        size_t nw = 0;
        if (l.op == HE_CONV2D) nw = (size_t)l.ch_out * l.ch_in * l.k * l.k;
        if (l.op == HE_CONV1D) nw = (size_t)l.ch_out * l.ch_in * l.k;
        if (l.op == HE_FC) nw = (size_t)l.ch_out * l.ch_in;
        if (nw) {
            if (!l.w || !l.b) throw HeError(HE_EINVAL, "layer weights missing");
            s.w.assign(l.w, l.w + nw);
            s.b.assign(l.b, l.b + l.ch_out);
        }
        if (l.op < HE_CONV2D || l.op > HE_APPROX_RELU) throw HeError(HE_EINVAL, "unknown layer op");
        out.push_back(std::move(s));
    }
    (void)Hi;
    return out;
}

static Feat run_layers(Ctx *c, Feat f, const std::vector<LayerSpec> &ls, PtCache *pc) {
    static const char *opname[] = {"?", "conv2d", "conv1d", "square", "avgpool", "flatten", "fc", "approx_relu"};
    for (size_t i = 0; i < ls.size(); ++i) {
        const LayerSpec &s = ls[i];
        std::string key = fmt("L%zu", i);
        c->prof_tag = fmt("%zu%s", i, opname[s.op <= HE_APPROX_RELU ? s.op : 0]);
        switch (s.op) {
            case HE_CONV2D: f = layer_conv(c, f, s, s.k, s.k, false, pc, key); break;
            case HE_CONV1D: f = layer_conv(c, f, s, 1, s.k, false, pc, key); break;
            case HE_SQUARE: f = layer_square(c, f); break;
            case HE_APPROX_RELU: f = layer_approx_relu(c, f, pc, key); break;
            case HE_AVGPOOL: f = layer_avgpool(c, f, s.k); break;
            case HE_FLATTEN: f = layer_flatten(c, f, pc, key); break;
            case HE_FC:
                if (f.x.lay.prev != PREV_FLAT && f.x.lay.prev != PREV_FC) f = layer_flatten(c, f, pc, key + "f");
                f = layer_fc(c, f, s, pc, key);
                break;
        }
    }
    c->prof_tag.clear();
    return f;
}

// ------------------------------------------------------------------ model
void model_check_input(const he_model *m, const Cts &x) {
    const Layout &L = x.lay;
    if (L.W_img != m->W_img || L.H_img != m->H_img || L.n_samples != m->spc || L.stride < m->plan.stride ||
        L.prev != PREV_INPUT || L.C != m->plan.C)
        throw HeError(HE_EINVAL, "ciphertext layout does not match the model");
    if (x.lp < m->plan.levels + 1) throw HeError(HE_ELEVEL, "not enough levels for this model");
}

// the schedule a model was compiled with, for the duration of one of its runs
struct ScheduleScope {
    Ctx *c;
    bool saved;
    ScheduleScope(Ctx *cx, bool literal) : c(cx), saved(cx->literal) { c->literal = literal; }
    ~ScheduleScope() { c->literal = saved; }
};

Cts model_infer(he_model *m, const Cts &x_in, bool use_graph) {
    Ctx *c = m->c;
    model_check_input(m, x_in);
    ScheduleScope sched(c, m->literal);
    // Drop-Level (Sec. IV-A): a ciphertext with more levels than the model consumes
    // loses its top limbs first, so every layer runs on the fewest limbs
    const Cts x = ct_drop_to(c, x_in, m->plan.levels + 1);
    Feat f;
    f.x = x;
    f.CH = 1;
    f.B = x.B;
    if (!use_graph) return run_layers(c, f, m->layers, &m->pc).x;
    std::string key = fmt("%u:%u:%.17g", x.B, x.lp, x.scale);
    auto it = m->graphs.find(key);
    const size_t inw = (size_t)x.B * cts_ct_words(c, x.lp);
    if (it == m->graphs.end()) {
        // the first time: an eager run fills the plaintext cache (the masks depend on the
        // layout, not on the batch size); then a warm run in the private pool and the capture
        if (!m->pc_filled) {
            run_layers(c, f, m->layers, &m->pc);
            m->pc_filled = true;
        }
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        ModelGraph g;
        c->active = &m->gpool;
        try {
            g.in = cts_alloc(c, x.B, x.lp, x.scale, x.lay);
            Feat fi = f;
            fi.x = g.in;
            {   // warm the private pool with one run of the same shapes
                Feat w = run_layers(c, fi, m->layers, &m->pc);
            }
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            const bool prof = c->profiling;
            c->profiling = false;   // no event records inside the graph
            const u64 before = c->launches;
            CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
            set_capturing(true);
            Feat r;
            try {
                r = run_layers(c, fi, m->layers, &m->pc);
            } catch (...) {
                set_capturing(false);
                cudaGraph_t tmpg = nullptr;
                cudaStreamEndCapture(c->stream, &tmpg);
                if (tmpg) cudaGraphDestroy(tmpg);
                c->profiling = prof;
                throw;
            }
            set_capturing(false);
            c->profiling = prof;
            g.kernels = c->launches - before;
            c->launches = before;
            CUDA_TRY(cudaStreamEndCapture(c->stream, &g.graph));
            CUDA_TRY(cudaGraphInstantiate(&g.exec, g.graph, 0));
            g.out = r.x;   // keeps the output buffer alive in the private pool
        } catch (...) {
            c->active = nullptr;
            throw;
        }
        c->active = nullptr;
        it = m->graphs.emplace(key, std::move(g)).first;
    }
    ModelGraph &g = it->second;
    CUDA_TRY(cudaMemcpyAsync(g.in.data(), x.data(), inw * 8, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaGraphLaunch(g.exec, c->stream));
    c->launches += g.kernels;
    Cts o = cts_alloc(c, g.out.B, g.out.lp, g.out.scale, g.out.lay);
    CUDA_TRY(cudaMemcpyAsync(o.data(), g.out.data(), (size_t)g.out.B * cts_ct_words(c, g.out.lp) * 8,
                             cudaMemcpyDeviceToDevice, c->stream));
    return o;
}

// ------------------------------------------------------------------ C ABI
static thread_local std::string g_err;

// the message he_last_error() returns on this thread (entry points of every translation unit)
const char *set_last_error(const char *msg) {
    g_err = msg;
    return g_err.c_str();
}

template <class F>
static he_status guard(F &&f) {
    try {
        f();
        return HE_OK;
    } catch (const HeError &e) {
        g_err = e.what();
        return e.code;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return HE_ENOMEM;
    } catch (const std::exception &e) {
        g_err = e.what();
        return HE_EINVAL;
    }
}

static Ctx *CX(he_ctx *h) {
    if (!h || !h->c) throw HeError(HE_EINVAL, "null context");
    CUDA_TRY(cudaSetDevice(h->c->device));
    return h->c.get();
}

he_ct *ct_wrap(Ctx *c, const Cts &x) {
    he_ct *h = new he_ct();
    h->keep = c->shared_from_this();
    h->c = c;
    h->x = x;
    return h;
}

static Feat gather_channels(Ctx *c, he_ct *const *in, u32 ch) {
    if (!in || !ch) throw HeError(HE_EINVAL, "no input channels");
    for (u32 i = 0; i < ch; ++i)
        if (!in[i]) throw HeError(HE_EINVAL, "null ciphertext");
    const Cts &a = in[0]->x;
    for (u32 i = 1; i < ch; ++i) {
        const Cts &b = in[i]->x;
        if (b.B != a.B || b.lp != a.lp) throw HeError(HE_EINVAL, "channels differ in batch or level");
        if (b.scale != a.scale) throw HeError(HE_ESCALE, "channels differ in scale");
    }
    Feat f;
    f.CH = ch;
    f.B = a.B;
    if (ch == 1) {
        f.x = a;
        return f;
    }
    f.x = cts_alloc(c, ch * a.B, a.lp, a.scale, a.lay);
    const size_t w = (size_t)a.B * cts_ct_words(c, a.lp);
    for (u32 i = 0; i < ch; ++i)
        CUDA_TRY(cudaMemcpyAsync(f.x.data() + i * w, in[i]->x.data(), w * 8, cudaMemcpyDeviceToDevice, c->stream));
    return f;
}

static void scatter_channels(Ctx *c, const Feat &f, he_ct **out) {
    for (u32 i = 0; i < f.CH; ++i) out[i] = ct_wrap(c, f.chan(c, i));
}

extern "C" {

const char *he_last_error(void) { return g_err.c_str(); }

he_status he_context_create(const he_params *p, he_ctx **out) {
    return guard([&] {
        if (!out) throw HeError(HE_EINVAL, "null output");
        Ctx *c = ctx_create(p);
        he_ctx *h = new he_ctx();
        h->c = std::shared_ptr<Ctx>(c, ctx_destroy);
        *out = h;
    });
}

void he_context_destroy(he_ctx *h) {
    if (!h) return;
    delete h;   // the context itself goes when its last ciphertext / model handle is freed
}

he_status he_context_primes(const he_ctx *h, uint64_t *out, size_t n) {
    return guard([&] {
        if (!h || !out || n < h->c->primes.size()) throw HeError(HE_EINVAL, "bad arguments");
        memcpy(out, h->c->primes.data(), h->c->primes.size() * 8);
    });
}

he_status he_keygen(he_ctx *h, const int32_t *steps, size_t n) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (n && !steps) throw HeError(HE_EINVAL, "null steps");
        keygen(c, std::vector<int>(steps, steps + n));
        c->naf = false;
    });
}

he_status he_context_set_schedule(he_ctx *h, uint32_t schedule) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (schedule != HE_SCHEDULE_FUSED && schedule != HE_SCHEDULE_LITERAL) throw HeError(HE_EINVAL, "unknown schedule");
        c->literal = schedule == HE_SCHEDULE_LITERAL;
    });
}

he_status he_keygen_pow2(he_ctx *h) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        std::vector<int> steps;
        for (u32 k = 1; k < c->N / 2; k *= 2) {
            steps.push_back((int)k);
            steps.push_back(-(int)k);
        }
        keygen(c, steps);
        c->naf = true;
    });
}

he_status he_encrypt(he_ctx *h, const double *x, int x_on_device, uint32_t W, uint32_t H, uint32_t nsamp,
                     uint32_t spc, uint32_t stride, uint64_t enc_seed, he_ct **out) {
    return he_encrypt_channels(h, x, x_on_device, 1, W, H, nsamp, spc, stride, enc_seed, out);
}

he_status he_encrypt_channels(he_ctx *h, const double *x, int x_on_device, uint32_t C, uint32_t W, uint32_t H,
                              uint32_t nsamp, uint32_t spc, uint32_t stride, uint64_t enc_seed, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!x || !out || !C || !W || !H || !nsamp) throw HeError(HE_EINVAL, "bad arguments");
        if (C > 1 && H == 1) throw HeError(HE_EINVAL, "several input channels need a 2-D image");
        const size_t len = (size_t)nsamp * C * W * H;
        const double *xd = x;
        DBuf tmp;
        if (!x_on_device) {
            tmp = DBuf(c, len);
            CUDA_TRY(cudaMemcpyAsync(tmp.p, x, len * 8, cudaMemcpyHostToDevice, c->stream));
            xd = reinterpret_cast<const double *>(tmp.p);
        }
        Cts ct = encrypt(c, xd, W, H, nsamp, spc, stride, enc_seed, C);
        if (!x_on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
        *out = ct_wrap(c, ct);
    });
}

he_status he_decrypt(he_ctx *h, const he_ct *ct, double *out, int out_on_device, size_t nper) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!ct || !out || !nper) throw HeError(HE_EINVAL, "bad arguments");
        const Cts &x = ct->x;
        if (nper > x.lay.stride && x.lay.n_samples > 1) throw HeError(HE_EINVAL, "n_per_sample above the stride");
        const size_t total = (size_t)x.B * x.lay.n_samples * nper;
        if (out_on_device) {
            decrypt_decode(c, out, x.data(), x.B, x.lp, x.scale, x.lay.stride, x.lay.n_samples, (u32)nper);
        } else {
            DBuf d(c, total);
            decrypt_decode(c, reinterpret_cast<double *>(d.p), x.data(), x.B, x.lp, x.scale, x.lay.stride,
                           x.lay.n_samples, (u32)nper);
            CUDA_TRY(cudaMemcpyAsync(out, d.p, total * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
        }
    });
}

he_status he_ct_info(const he_ct *ct, uint32_t *batch, uint32_t *limbs, double *scale) {
    return guard([&] {
        if (!ct) throw HeError(HE_EINVAL, "null ciphertext");
        if (batch) *batch = ct->x.B;
        if (limbs) *limbs = ct->x.lp;
        if (scale) *scale = ct->x.scale;
    });
}

he_status he_ct_layout(const he_ct *ct, uint32_t *spc, uint32_t *stride, uint32_t *interval) {
    return guard([&] {
        if (!ct) throw HeError(HE_EINVAL, "null ciphertext");
        if (spc) *spc = ct->x.lay.n_samples;
        if (stride) *stride = ct->x.lay.stride;
        if (interval) *interval = ct->x.lay.I;
    });
}

he_status he_ct_export(he_ctx *h, const he_ct *ct, uint64_t *coeff) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!ct || !coeff) throw HeError(HE_EINVAL, "bad arguments");
        const Cts &x = ct->x;
        const size_t w = (size_t)x.B * cts_ct_words(c, x.lp);
        DBuf t(c, w);
        CUDA_TRY(cudaMemcpyAsync(t.p, x.data(), w * 8, cudaMemcpyDeviceToDevice, c->stream));
        ntt_inverse(c, t.p, rows_regular(x.B * 2 * x.lp, x.lp, x.lp, 0));
        CUDA_TRY(cudaMemcpyAsync(coeff, t.p, w * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
}

void he_ct_free(he_ct *ct) {
    if (!ct) return;
    std::shared_ptr<Ctx> k = ct->keep;   // outlives the lock: the context may go with the handle
    CtxLock lk(k.get());
    delete ct;
}

he_status he_rotate(he_ctx *h, const he_ct *in, int32_t step, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out) throw HeError(HE_EINVAL, "bad arguments");
        *out = ct_wrap(c, ct_rotate(c, in->x, step));
    });
}

he_status he_rotate_hoisted(he_ctx *h, const he_ct *in, const int32_t *steps, size_t n, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out || !steps || !n) throw HeError(HE_EINVAL, "bad arguments");
        std::vector<Cts> r = ct_rotate_hoisted(c, in->x, std::vector<int>(steps, steps + n));
        for (size_t i = 0; i < n; ++i) out[i] = ct_wrap(c, r[i]);
    });
}

he_status he_drop_level(he_ctx *h, const he_ct *in, uint32_t levels, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out) throw HeError(HE_EINVAL, "bad arguments");
        if (levels >= in->x.lp) throw HeError(HE_ELEVEL, "drop level: not that many levels left");
        *out = ct_wrap(c, ct_drop_to(c, in->x, in->x.lp - levels));
    });
}

// Sec. III-B: input i rotated right by (sample positions before it) * stride, all added;
// one combination of the per-input rotations with a single ModDown
he_status he_pack(he_ctx *h, he_ct *const *in, uint32_t n, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out || !n) throw HeError(HE_EINVAL, "bad arguments");
        for (u32 i = 0; i < n; ++i)
            if (!in[i]) throw HeError(HE_EINVAL, "null ciphertext");
        const Layout &L0 = in[0]->x.lay;
        std::vector<int> steps;
        u64 off = 0;
        for (u32 i = 0; i < n; ++i) {
            const Cts &x = in[i]->x;
            const Layout &L = x.lay;
            if (x.B != 1) throw HeError(HE_EINVAL, "pack: every input must be one ciphertext");
            if (L.prev != PREV_INPUT || L.W_img != L0.W_img || L.H_img != L0.H_img || L.stride != L0.stride ||
                L.dims != L0.dims)
                throw HeError(HE_EINVAL, "pack: inputs differ in layout");
            steps.push_back(-(int)(off * L0.stride));
            off += L.n_samples;
        }
        if (off * L0.stride > c->N / 2) throw HeError(HE_ESLOTS, "pack: the samples do not fit in the slots");
        Feat f = gather_channels(c, in, n);
        Cts y = n > 1 ? ct_lincomb_diag(c, f.x, n, 1, steps) : f.x;
        y.lay = L0;
        y.lay.n_samples = (u32)off;
        *out = ct_wrap(c, y);
    });
}

he_status he_rescale(he_ctx *h, const he_ct *in, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out) throw HeError(HE_EINVAL, "bad arguments");
        *out = ct_wrap(c, ct_rescale(c, in->x));
    });
}

he_status he_mul_plain(he_ctx *h, const he_ct *in, const double *v, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !out || !v) throw HeError(HE_EINVAL, "bad arguments");
        const u32 M = c->N / 2;
        Layout one = in->x.lay;
        one.stride = M;
        one.n_samples = 1;
        std::vector<u32> off{0}, pos;
        std::vector<double> val;
        for (u32 j = 0; j < M; ++j)
            if (v[j] != 0.0) {
                pos.push_back(j);
                val.push_back(v[j]);
            }
        off.push_back((u32)pos.size());
        std::vector<DBuf> tmp;
        const u64 *pt = get_pts(c, nullptr, "mulplain", tmp, one, off, pos, val, c->scale, in->x.lp);
        *out = ct_wrap(c, ct_mul_pt(c, in->x, pt, c->scale));
    });
}

he_status he_add(he_ctx *h, const he_ct *a, const he_ct *b, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!a || !b || !out) throw HeError(HE_EINVAL, "bad arguments");
        *out = ct_wrap(c, ct_add(c, a->x, b->x));
    });
}

he_status he_square(he_ctx *h, he_ct *const *in, uint32_t n, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!out) throw HeError(HE_EINVAL, "bad arguments");
        Feat f = gather_channels(c, in, n);
        scatter_channels(c, layer_square(c, f), out);
    });
}

he_status he_approx_relu(he_ctx *h, he_ct *const *in, uint32_t n, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!out) throw HeError(HE_EINVAL, "bad arguments");
        Feat f = gather_channels(c, in, n);
        scatter_channels(c, layer_approx_relu(c, f, nullptr, "approx_relu"), out);
    });
}

static he_status conv_common(he_ctx *h, he_ct *const *in, uint32_t ci, const double *w, const double *bias,
                             uint32_t co, uint32_t K, uint32_t S, int incremental, he_ct **out, bool two_d) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!w || !bias || !out || !co || !K || !S) throw HeError(HE_EINVAL, "bad arguments");
        Feat f = gather_channels(c, in, ci);
        LayerSpec s;
        s.op = two_d ? HE_CONV2D : HE_CONV1D;
        s.ci = ci;
        s.co = co;
        s.k = K;
        s.s = S;
        size_t nw = (size_t)co * ci * K * (two_d ? K : 1);
        s.w.assign(w, w + nw);
        s.b.assign(bias, bias + co);
        u32 kh = two_d ? K : 1;
        std::vector<int> need;
        for (u32 j = 0; j < kh; ++j)
            for (u32 k = 0; k < K; ++k)
                if (!incremental) require_key(c, (int)(f.x.lay.I * (k + f.x.lay.W_img * j)));
        Feat r = layer_conv(c, f, s, kh, K, incremental != 0, nullptr, "conv");
        scatter_channels(c, r, out);
    });
}

he_status he_conv2d(he_ctx *h, he_ct *const *in, uint32_t ci, const double *w, const double *bias, uint32_t co,
                    uint32_t K, uint32_t S, int incremental, he_ct **out) {
    return conv_common(h, in, ci, w, bias, co, K, S, incremental, out, true);
}

he_status he_conv1d(he_ctx *h, he_ct *const *in, uint32_t ci, const double *w, const double *bias, uint32_t co,
                    uint32_t K, uint32_t S, int incremental, he_ct **out) {
    return conv_common(h, in, ci, w, bias, co, K, S, incremental, out, false);
}

he_status he_avgpool(he_ctx *h, he_ct *const *in, uint32_t ch, uint32_t cc, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!out || !cc) throw HeError(HE_EINVAL, "bad arguments");
        Feat f = gather_channels(c, in, ch);
        scatter_channels(c, layer_avgpool(c, f, cc), out);
    });
}

he_status he_flatten(he_ctx *h, he_ct *const *in, uint32_t ch, he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!out) throw HeError(HE_EINVAL, "bad arguments");
        Feat f = gather_channels(c, in, ch);
        *out = ct_wrap(c, layer_flatten(c, f, nullptr, "flatten").x);
    });
}

he_status he_fc(he_ctx *h, const he_ct *in, const double *Wm, const double *b, uint32_t din, uint32_t dout,
                he_ct **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!in || !Wm || !b || !out || !din || !dout) throw HeError(HE_EINVAL, "bad arguments");
        LayerSpec s;
        s.op = HE_FC;
        s.ci = din;
        s.co = dout;
        s.w.assign(Wm, Wm + (size_t)din * dout);
        s.b.assign(b, b + dout);
        Feat f;
        f.x = in->x;
        f.CH = 1;
        f.B = in->x.B;
        *out = ct_wrap(c, layer_fc(c, f, s, nullptr, "fc").x);
    });
}

he_status he_model_plan(const he_layer *layers, size_t n, uint32_t Wi, uint32_t Hi, uint32_t *stride,
                        uint32_t *levels, int32_t *steps, size_t *n_steps) {
    return he_model_plan_schedule(layers, n, Wi, Hi, HE_SCHEDULE_FUSED, stride, levels, steps, n_steps);
}

he_status he_model_plan_schedule(const he_layer *layers, size_t n, uint32_t Wi, uint32_t Hi, uint32_t schedule,
                                 uint32_t *stride, uint32_t *levels, int32_t *steps, size_t *n_steps) {
    return guard([&] {
        if (!layers || !n || !Wi || !Hi) throw HeError(HE_EINVAL, "bad arguments");
        if (schedule != HE_SCHEDULE_FUSED && schedule != HE_SCHEDULE_LITERAL) throw HeError(HE_EINVAL, "unknown schedule");
        Plan p = plan_layers(copy_layers(layers, n, Hi), Wi, Hi, schedule == HE_SCHEDULE_LITERAL);
        if (stride) *stride = p.stride;
        if (levels) *levels = p.levels;
        if (n_steps) {
            if (steps) {
                if (*n_steps < p.steps.size()) throw HeError(HE_EINVAL, "steps buffer too small");
                for (size_t i = 0; i < p.steps.size(); ++i) steps[i] = p.steps[i];
            }
            *n_steps = p.steps.size();
        }
    });
}

he_status he_model_compile(he_ctx *h, const he_layer *layers, size_t n, uint32_t Wi, uint32_t Hi, uint32_t spc,
                           he_model **out) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!layers || !n || !out || !spc) throw HeError(HE_EINVAL, "bad arguments");
        std::unique_ptr<he_model> m(new he_model());
        m->gpool.graph = true;   // the model's graphs run one at a time on its context's stream
        m->keep = c->shared_from_this();
        m->c = c;
        m->layers = copy_layers(layers, n, Hi);
        m->W_img = Wi;
        m->H_img = Hi;
        m->spc = spc;
        m->literal = c->literal;
        m->plan = plan_layers(m->layers, Wi, Hi, m->literal);
        if ((u64)m->plan.stride * spc > c->N / 2) throw HeError(HE_ESLOTS, "samples do not fit in the slots");
        if (m->plan.levels + 1 > c->L1) throw HeError(HE_ELEVEL, "the modulus chain is too short for this model");
        for (int s : m->plan.steps) {
            if (!c->naf) {
                require_key(c, s);
                continue;
            }
            for (int t : naf_terms(s, c->N / 2)) require_key(c, t);
        }
        *out = m.release();
    });
}

he_status he_infer(he_model *m, const he_ct *in, int use_graph, he_ct **out) {
    return guard([&] {
        if (!m || !in || !out) throw HeError(HE_EINVAL, "bad arguments");
        Ctx *c = m->c;
        CtxLock lk(c);
        CUDA_TRY(cudaSetDevice(c->device));
        *out = ct_wrap(c, model_infer(m, in->x, use_graph != 0));
    });
}

he_status he_model_set_mask_budget(he_model *m, uint64_t bytes) {
    return guard([&] {
        if (!m) throw HeError(HE_EINVAL, "null model");
        CtxLock lk(m->c);
        m->pc.mask_budget = (size_t)bytes;
    });
}

void he_model_free(he_model *m) {
    if (!m) return;
    std::shared_ptr<Ctx> k = m->keep;
    CtxLock lk(k.get());
    cudaSetDevice(m->c->device);
    cudaStreamSynchronize(m->c->stream);
    delete m;
}

he_status he_ntt(he_ctx *h, uint64_t *data, uint32_t n_limbs, const uint32_t *prime_idx, int inverse) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        if (!data || !prime_idx || !n_limbs) throw HeError(HE_EINVAL, "bad arguments");
        std::vector<u32> rows;
        for (u32 i = 0; i < n_limbs; ++i) {
            if (prime_idx[i] >= c->nprimes()) throw HeError(HE_EINVAL, "prime index out of range");
            rows.push_back((i << 8) | prime_idx[i]);
        }
        std::string key = "user";
        for (u32 i = 0; i < n_limbs; ++i) key += fmt(":%u", prime_idx[i]);
        RowSet rs = rows_list(c, key, rows);
        if (inverse)
            ntt_inverse(c, data, rs);
        else
            ntt_forward(c, data, rs);
    });
}

he_status he_sync(he_ctx *h) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
}

uint64_t he_kernel_launches(const he_ctx *h) { return h && h->c ? h->c->launches : 0; }

he_status he_profile_begin(he_ctx *h) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        c->recs.clear();
        c->profiling = true;
    });
}

he_status he_profile_end(he_ctx *h, he_kernel_stat *out, size_t cap, size_t *n) {
    return guard([&] {
        Ctx *c = CX(h);
        CtxLock lk_(c);
        c->profiling = false;
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        std::map<std::string, he_kernel_stat> agg;
        std::vector<std::string> order;
        for (auto &r : c->recs) {
            float ms = 0;
            CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
            const std::string key = r.tag.empty() ? std::string(r.name) : r.tag + "/" + r.name;
            auto it = agg.find(key);
            if (it == agg.end()) {
                he_kernel_stat s;
                memset(&s, 0, sizeof s);
                strncpy(s.name, key.c_str(), sizeof s.name - 1);
                it = agg.emplace(key, s).first;
                order.push_back(key);
            }
            it->second.launches++;
            it->second.total_ms += ms;
            it->second.bytes += r.bytes;
            it->second.ops += r.ops;
            c->ev_free.push_back(r.a);
            c->ev_free.push_back(r.b);
        }
        c->recs.clear();
        if (n) *n = order.size();
        if (out)
            for (size_t i = 0; i < order.size() && i < cap; ++i) out[i] = agg[order[i]];
    });
}

}  // extern "C"
