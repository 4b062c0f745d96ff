// keyswitch.cuh -- hybrid key switching and rescale (keyswitch.cu).
#pragma once
#include "he_internal.cuh"
#include "ring.cuh"

#define KEYLIST_MAX 64
// a single-output weighted combination of one channel folds its weights into the keys from this
// many ciphertexts on
#define COMB_FOLD_MIN_B 16
// Per rotation step s of one launch: the switching key [dnum][2][L+1+K][N] and
// the Galois element applied to the ModUp'ed digits (1 = none); for the
// pre-permuted form, ginv is the inverse Galois element g^{-1} mod 2N.
struct KeyList {
    const u64 *key[KEYLIST_MAX];    // K_{g,j}
    const u64 *keyp[KEYLIST_MAX];   // K'_{g,j} = sigma_g^{-1}(K_{g,j}) (Galois keys only)
    u32 g[KEYLIST_MAX];
    u32 ginv[KEYLIST_MAX];
};

void keyswitch_init(Ctx *c);
u32 ks_digits(const Ctx *c, u32 lp);
void ks_modup(Ctx *c, u64 *D, const u64 *xe, size_t xe_bstride, u32 B, u32 lp);
void ks_inner(Ctx *c, u64 *acc, const u64 *D, const KeyList &kl, u32 S, u32 B, u32 lp, const u64 *padd = nullptr,
              size_t padd_bstride = 0);
void ks_lazy(Ctx *c, u64 *acc, const u64 *D, const u64 *x, const KeyList &kl, u32 S, u32 B, u32 lp);
void ks_comb(Ctx *c, u64 *Z, const u64 *D, const u64 *x, const KeyList &kl, u32 S, u32 CH, u32 B, u32 lp,
             const u64 *w, u32 O, size_t w_ostride, int accumulate);
void ks_moddown(Ctx *c, u64 *out, u64 *acc, const u64 *addend, size_t addend_bstride, u32 add_mask,
                const KeyList &kl, u32 S, u32 B, u32 lp);
void rescale_batch(Ctx *c, u64 *out, const u64 *in, u32 B, u32 lp);
void ks_moddown_rescale(Ctx *c, u64 *out, u64 *acc, u32 nct, u32 lp);
