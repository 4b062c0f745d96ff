// ops.cuh -- host-side ciphertext operations of libunihenn (he.cu, encode.cu).
#pragma once
#include "he_internal.cuh"
#include "keyswitch.cuh"
#include "ring.cuh"

// the C handle of a context (shared by its ciphertext and model handles)
struct he_ctx {
    std::shared_ptr<Ctx> c;
};

// A ciphertext batch that may be a view into a larger buffer
struct Cts {
    std::shared_ptr<DBuf> mem;
    size_t off = 0;          // words
    u32 B = 0, lp = 0;
    double scale = 1.0;
    Layout lay;
    u64 *data() const { return mem->p + off; }
};

Cts cts_alloc(Ctx *c, u32 B, u32 lp, double scale, const Layout &lay);
Cts cts_view(const Cts &base, size_t off_words, u32 B);
size_t cts_ct_words(const Ctx *c, u32 lp);    // words of one ciphertext: 2*lp*N

// context set-up (he.cu)
Ctx *ctx_create(const he_params *p);
void ctx_destroy(Ctx *c);
void keygen(Ctx *c, const std::vector<int> &steps);

// encode.cu
void encode_init(Ctx *c);
void encode_dense(Ctx *c, u64 *out, const double *z, u32 nv, double scale, u32 lp, bool check);
void encode_sparse_dev(Ctx *c, u64 *out, const u32 *off, u32 nv, const u32 *pos, const double *val, u32 stride,
                       u32 ns, double scale, u32 lp, u32 ext);
void encode_sparse(Ctx *c, u64 *out, const std::string &key, const std::vector<u32> &off,
                   const std::vector<u32> &pos, const std::vector<double> &val, u32 stride, u32 ns, double scale,
                   u32 lp, u32 ext = 0);
void check_encode_errors(Ctx *c);
void pack_samples(Ctx *c, double *z, const double *x, u32 nsamp, u32 spc, u32 stride, u32 len, u32 nct);
void enc_combine(Ctx *c, u64 *ct, const u64 *u, const u64 *me, const u64 *e1, u32 lp, u32 B);
void decrypt_decode(Ctx *c, double *out, const u64 *ct, u32 B, u32 lp, double scale, u32 stride, u32 ns, u32 nper);

// he.cu
Cts encrypt(Ctx *c, const double *x_dev, u32 W, u32 H, u32 nsamp, u32 spc, u32 stride, u64 enc_seed, u32 C = 1);
Cts ct_add(Ctx *c, const Cts &a, const Cts &b);
void ct_add_inplace(Ctx *c, Cts &a, const Cts &b);
Cts ct_rescale(Ctx *c, const Cts &a);
Cts ct_drop_level(Ctx *c, const Cts &a);
// linear combinations of rotations evaluated rotate-then-multiply, one rotation at a time:
// with power-of-two keys (chains) and in the paper-order schedule (direct rotations)
inline bool seq_lincomb(const Ctx *c) { return c->naf || c->literal; }
// limbs beyond Q_l that the plaintexts of ct_lincomb carry: K (hoisted, over Q_l u P), or 0
// when combinations are rotate-then-multiply (over Q_l)
inline u32 ks_ext(const Ctx *c) { return seq_lincomb(c) ? 0 : c->K; }
// a rotation step as the signed powers of two of its non-adjacent form, lowest first
std::vector<int> naf_terms(int64_t r, u32 slots);
Cts ct_drop_to(Ctx *c, const Cts &a, u32 keep);
Cts ct_rotate(Ctx *c, const Cts &a, int step);
// Rotations of one batch by several steps sharing one ModUp.  out[i] = Rot(a, steps[i]).
// All outputs live in one buffer, step i at offset i*B*2*lp*N (the layout the MAC reads).
std::vector<Cts> ct_rotate_hoisted(Ctx *c, const Cts &a, const std::vector<int> &steps);
void ct_rotate_hoisted_into(Ctx *c, const Cts &a, const std::vector<int> &steps, u64 *out);
Cts ct_square(Ctx *c, const Cts &a);
// with rescale every output is also rescaled: ModDown and rescale as one division by q_top * P
Cts ct_lincomb(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<int> &steps, const u64 *pts, u32 O,
               double pt_scale, bool rescale = false);
Cts ct_lincomb_diag(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<int> &steps);
Cts ct_lincomb_chan(Ctx *c, const Cts &X, u32 CH, u32 B, const std::vector<std::vector<int>> &steps, const u64 *pts,
                    double pt_scale, bool rescale);
Cts ct_mul_pt(Ctx *c, const Cts &a, const u64 *pt, double pt_scale);
void ct_add_pt_inplace(Ctx *c, Cts &a, const u64 *pt);
void require_key(Ctx *c, int step);
