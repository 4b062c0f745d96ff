// ring.cuh -- declarations of the elementwise ring kernels (ring.cu).
#pragma once
#include "he_internal.cuh"

enum { OP_ADD = 0, OP_SUB = 1, OP_MUL = 2, OP_NEG = 3 };

#define SEEDLIST_MAX 64
struct SeedList {
    u64 seed[SEEDLIST_MAX];
    u64 stream[SEEDLIST_MAX];
};

void ew_binop(Ctx *c, int op, u64 *out, const u64 *a, const u64 *b, u32 rows, u32 period, u32 lp, u32 pbase);
void ew_bcast(Ctx *c, int op, u64 *out, const u64 *a, const u64 *pt, u32 B, u32 lp, u32 kmask);
void add_plain_multi(Ctx *c, u64 *out, const u64 *pt, u32 O, u32 B, u32 lp, size_t o_stride);
void galois_permute(Ctx *c, u64 *out, const u64 *in, u32 rows, u32 g);
void tensor_square(Ctx *c, u64 *d, const u64 *a, u32 B, u32 lp);
void sample_small(Ctx *c, u64 *out, const SeedList &sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase, int kind);
void sample_uniform(Ctx *c, u64 *out, const SeedList &sl, u32 nvec, u32 rows, u32 period, u32 lp, u32 pbase);
void mac_tc_init();   // once per context: the tensor-core MAC's shared-memory limit
void mac(Ctx *c, u64 *out, size_t out_ostride, const u64 *x, size_t x_tstride, const u64 *pt, u32 O, u32 T, u32 B,
         u32 lp, u32 lpq = ~0u, u32 pbase = 0, int accumulate = 0, size_t pt_ostride = 0);
// out[r] (+)= sum_{s<S} a[s*stride_words + r*N ...] over rows r < nrows, prime map (period, lp, pbase)
void sum_stack(Ctx *c, u64 *out, const u64 *a, size_t stride_words, u32 S, u32 nrows, u32 period, u32 lp, u32 pbase,
               int accumulate);
void gather_rows(Ctx *c, u64 *out, const u64 *in, u32 nrows, size_t stride_rows);
