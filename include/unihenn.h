/*
 * unihenn.h -- C ABI of the GB300 (sm_103a) library for UniHENN's encrypted
 * CNN inference (Choi et al., "UniHENN: Designing Faster and More Versatile
 * Homomorphic Encryption-based CNNs without im2col", arXiv 2402.03060).
 *
 * Every ring operation behind these calls runs as a CUDA kernel of
 * libunihenn.so; no call has a CPU fallback.  Arguments are plain pointers
 * and sizes.  Conventions for every entry point:
 *   - the return value is a he_status; on failure he_last_error() gives a
 *     thread-local message and no output handle is written;
 *   - handles (he_ctx, he_ct, he_model) are allocated by the library and freed
 *     by the caller with the matching *_free / *_destroy call;
 *   - input arrays are borrowed for the duration of the call only;
 *   - work is queued on the context's stream; calls that return data to host
 *     memory (he_decrypt with a host buffer, he_ct_export, he_context_primes)
 *     synchronise that stream before returning.
 *
 * Ciphertext layout in device memory: a he_ct is a BATCH of B ciphertexts of
 * the same level, scale and slot layout, stored contiguously as
 * [B][2][L'][N] uint64 residues (c0 then c1, limbs q_0..q_{L'-1}), evaluation
 * form in bit-reversed order.  The slot layout is the paper's flattened
 * single-ciphertext layout (Sec. III-A): sample k of a ciphertext occupies
 * slots k*stride ... (Sec. III-B), value (r, c) of a feature map at
 * I*(r*W_img + c) with I the interval (Sec. IV-B, V-A).
 */
#ifndef UNIHENN_H
#define UNIHENN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HE_OK = 0,
    HE_EINVAL = 1,     /* bad argument (null pointer, size out of range, shape mismatch) */
    HE_ENOMEM = 2,     /* device allocation failed */
    HE_ELEVEL = 3,     /* not enough levels left for the operation (paper Sec. II-B "depth") */
    HE_ESCALE = 4,     /* operands of an addition have different scales */
    HE_ESLOTS = 5,     /* the slot layout does not fit in N/2 slots (paper Sec. V) */
    HE_ENOKEY = 6,     /* a rotation needs a Galois key that he_keygen did not create */
    HE_ECUDA = 7,      /* a CUDA call or kernel failed */
    HE_ETIMEOUT = 8,   /* a bounded device wait ran out */
    HE_EOVERFLOW = 9   /* an encoded coefficient does not fit in 63 bits (scale too large) */
} he_status;

typedef struct he_ctx he_ctx;
typedef struct he_ct he_ct;
typedef struct he_model he_model;

/* CKKS parameters (paper Sec. VI-D, Table II: slots, scale, modulus chain, depth).
 * The modulus chain is the n_data data primes followed by n_special special
 * primes; prime i is the largest prime below 2^prime_bits[i] that is 1 mod 2N
 * and not used by an earlier entry.  Hybrid key switching uses dnum digits of
 * ceil(n_data/dnum) consecutive data primes.  Depth = n_data - 1. */
typedef struct {
    uint32_t log2n;              /* N = 2^log2n; 4 <= log2n <= 15 */
    uint32_t n_data;             /* data primes (L+1), 1..32 */
    uint32_t n_special;          /* special primes K, 1..4 */
    const uint32_t *prime_bits;  /* n_data + n_special bit sizes, each 20..60 */
    uint32_t dnum;               /* 1..min(n_data, 16), with ceil(n_data/dnum) <= 8 */
    double log2_scale;           /* Delta = 2^log2_scale */
    uint64_t seed;               /* key-generation seed (counter-based SplitMix64) */
    int device;                  /* CUDA device ordinal */
    void *stream;                /* cudaStream_t to queue on; NULL = library-owned stream */
} he_params;

/* Create a context: primes, NTT/FFT tables and the device memory pool.
 * Errors: HE_EINVAL (parameters out of range), HE_ECUDA, HE_ENOMEM. */
he_status he_context_create(const he_params *p, he_ctx **out);
void he_context_destroy(he_ctx *ctx);

/* Copy the modulus chain (data primes, then special primes) to host out[n]. */
he_status he_context_primes(const he_ctx *ctx, uint64_t *out, size_t n);

/* Generate the secret key (kept on the device), the public key, the
 * relinearisation key and one Galois key per rotation step in rot_steps
 * (Rot(v, r) moves slot j+r to slot j, paper Sec. II-B; negative r rotates
 * right).  Key sizes: each switching key is dnum*2*(n_data+n_special)*N words.
 * Errors: HE_EINVAL, HE_ENOMEM, HE_ECUDA. */
he_status he_keygen(he_ctx *ctx, const int32_t *rot_steps, size_t n_steps);

/* he_keygen with the power-of-two Galois key set, the key set the paper's SEAL
 * setup uses: keys for the steps +-2^k (2^k < N/2) only, 2*log2(N/2) keys in
 * place of one per distinct step.  From then on every rotation is the chain of
 * rotations of its step's non-adjacent form (Reitwiesner), lowest power first,
 * chains of one input sharing their common prefixes, and each linear combination
 * of rotations is evaluated as rotate-then-multiply over Q_l followed by the
 * rescale (more key switches, far less key memory).  he_keygen returns the
 * context to one key per step.  Errors: HE_ENOMEM, HE_ECUDA. */
he_status he_keygen_pow2(he_ctx *ctx);

/* Evaluation schedule of the layer calls on this context and of the models compiled on it
 * from then on (a compiled model keeps the schedule it was compiled with).
 *   HE_SCHEDULE_FUSED (0, the default): the rotations of one input share one ModUp
 *     (hoisting); a linear combination of rotations (convolution, pooling, the flatten's
 *     stages, FC, channel packing) is accumulated over Q_l u P with one ModDown per output;
 *     a ModDown followed by a rescale is one division by q_top * P; the flatten's last
 *     stage may be merged with the channel packing.  The same slot values as the literal
 *     schedule, other ciphertext bits (other key-switch and rescale rounding).
 *   HE_SCHEDULE_LITERAL (1): the paper's order, one operation at a time -- Algorithm 1
 *     (Sec. IV-B), the pooling of Sec. IV-C, the flatten steps of Sec. IV-E and Algorithm 2
 *     (Sec. IV-D) as listed: every Rot is its own key switch (ModUp, inner product,
 *     ModDown, plus sigma_g(c0)), Mul (P) by the mask over Q_l, Add, then the centred
 *     rescale; square = tensor, relinearise (ModDown), rescale; a flatten stage multiplies
 *     the masks first and rotates the products; the channel packing follows the last
 *     stage.  Its models need the steps he_model_plan_schedule gives for it.
 * Errors: HE_EINVAL (unknown schedule). */
enum { HE_SCHEDULE_FUSED = 0, HE_SCHEDULE_LITERAL = 1 };
he_status he_context_set_schedule(he_ctx *ctx, uint32_t schedule);

/* Flatten and encrypt (paper Sec. III-A/B): x is [n_samples][H][W] doubles,
 * host memory (x_on_device = 0) or device memory (1).  Sample k goes to
 * ciphertext k / samples_per_ct at slot offset (k % samples_per_ct)*stride,
 * row-major, zero elsewhere.  Ciphertext b is a public-key encryption at the
 * top level with randomness seeded by enc_seed + b.  *out is a batch of
 * ceil(n_samples / samples_per_ct) ciphertexts whose layout records
 * (W_img = W, H_img = H, stride, samples_per_ct).
 * Errors: HE_EINVAL, HE_ESLOTS (samples_per_ct*stride > N/2 or W*H > stride),
 * HE_EOVERFLOW, HE_ECUDA. */
he_status he_encrypt(he_ctx *ctx, const double *x, int x_on_device, uint32_t W, uint32_t H,
                     uint32_t n_samples, uint32_t samples_per_ct, uint32_t stride,
                     uint64_t enc_seed, he_ct **out);

/* he_encrypt for samples of C channels, x [n_samples][C][H][W]: each sample is
 * flattened channel-major, row-major (Sec. III-A), value (i, r, c) at slot
 * offset i*W*H + r*W + c of its position; C*W*H <= stride.  A model whose first
 * convolution has CH_in = C reads input channel i through an extra rotation by
 * i*W*H.  C = 1 is he_encrypt.  Errors as he_encrypt; HE_EINVAL for C > 1 with
 * H = 1. */
he_status he_encrypt_channels(he_ctx *ctx, const double *x, int x_on_device, uint32_t C, uint32_t W, uint32_t H,
                              uint32_t n_samples, uint32_t samples_per_ct, uint32_t stride, uint64_t enc_seed,
                              he_ct **out);

/* Decrypt and decode (paper Sec. III, Fig. 1: the client decrypts the encrypted
 * result with its secret key and reads its values from the slots; decoding is the
 * canonical-embedding inverse of he_encrypt's encoding, Sec. II-B).
 * out is [B*samples_per_ct][n_per_sample] doubles (host or
 * device), the slots k*stride + [0, n_per_sample) of every sample position.
 * Decoding reads limb q_0, valid while |message * scale| < q_0/2.
 * Errors: HE_EINVAL, HE_ECUDA. */
he_status he_decrypt(he_ctx *ctx, const he_ct *ct, double *out, int out_on_device, size_t n_per_sample);

/* Batch combining (paper Sec. III-B), a client-side step: n ciphertexts, each a
 * batch of one in the input layout of the same image size and stride (as
 * he_encrypt makes them), become one ciphertext.  Input i is rotated right by
 * s_i * stride, s_i = the sample positions of the inputs before it, and all are
 * added: one key switch per input after the first, summed over Q u P with a
 * single ModDown.  The result's layout has the sum of the inputs' sample
 * positions.  Needs the Galois keys of the steps -s_i*stride.  *out is a new
 * handle.  Errors: HE_EINVAL (null, batch != 1, layouts differ), HE_ESLOTS
 * (the samples do not fit in N/2 slots), HE_ESCALE / HE_EINVAL (scale or level
 * differ), HE_ENOKEY. */
he_status he_pack(he_ctx *ctx, he_ct *const *in, uint32_t n, he_ct **out);

/* Drop-Level (paper Sec. IV-A) as a modulus drop: the top `levels` limbs of
 * every polynomial are removed; message, scale and layout are unchanged (levels
 * = 0 gives a new handle on the same data).  he_infer applies it by itself to an
 * input with more levels than the model consumes.  *out is a new handle.
 * Errors: HE_EINVAL, HE_ELEVEL (fewer than levels + 1 limbs). */
he_status he_drop_level(he_ctx *ctx, const he_ct *in, uint32_t levels, he_ct **out);

/* Batch size, active limbs L' and scale of a ciphertext batch. */
he_status he_ct_info(const he_ct *ct, uint32_t *batch, uint32_t *limbs, double *scale);

/* Slot layout of a ciphertext batch: sample positions per ciphertext, slots
 * per sample, and the interval I of the current feature map. */
he_status he_ct_layout(const he_ct *ct, uint32_t *samples_per_ct, uint32_t *stride, uint32_t *interval);

/* Copy a ciphertext batch to host memory in COEFFICIENT form,
 * [B][2][L'][N] uint64 (independent of the NTT ordering; used for parity). */
he_status he_ct_export(he_ctx *ctx, const he_ct *ct, uint64_t *coeff);
void he_ct_free(he_ct *ct);

/* ---- ciphertext operations (paper Sec. II-B) ---------------------------- */
/* Rot(ct, step) for every ciphertext of the batch: Galois automorphism and
 * hybrid key switching.  Errors: HE_ENOKEY, HE_ECUDA. */
he_status he_rotate(he_ctx *ctx, const he_ct *in, int32_t step, he_ct **out);
/* Several rotations of the same batch sharing one ModUp of c1 (hoisting);
 * out[i] receives Rot(in, steps[i]); a step of 0 (mod N/2) copies the input. */
he_status he_rotate_hoisted(he_ctx *ctx, const he_ct *in, const int32_t *steps, size_t n, he_ct **out);
/* Divide by the top prime (rescale); HE_ELEVEL at one limb. */
he_status he_rescale(he_ctx *ctx, const he_ct *in, he_ct **out);
/* Mul (P) by the slot vector v[N/2] (host) encoded at scale Delta; no rescale. */
he_status he_mul_plain(he_ctx *ctx, const he_ct *in, const double *v, he_ct **out);
/* Add (C); HE_ESCALE / HE_EINVAL on scale / level / batch mismatch. */
he_status he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
/* Mul (C) of each ciphertext by itself, relinearised and rescaled (square
 * activation, paper Sec. IV-F). */
he_status he_square(he_ctx *ctx, he_ct *const *in, uint32_t n, he_ct **out);
/* Approximate ReLU f(x) = 0.375373 + 0.5 x + 0.117071 x^2 (paper Sec. IV-F, model M3) on n
 * channel ciphertexts; 2 levels.  A pending average-pooling factor p is folded in as
 * f(p x) (Sec. IV-C).  The constant and the coefficients are applied at the layout's valid
 * slots only.  out[n] are new handles.  Errors: HE_ELEVEL (fewer than three limbs), HE_EINVAL. */
he_status he_approx_relu(he_ctx *ctx, he_ct *const *in, uint32_t n, he_ct **out);

/* ---- UniHENN layers (paper Sec. IV) on channel lists -------------------- */
/* Algorithm 1: in[ch_in] -> out[ch_out]; w [ch_out][ch_in][K][K] (conv2d) or
 * [ch_out][ch_in][K] (conv1d); bias [ch_out]; stride S.  incremental = 0:
 * rotations of each input share one ModUp; 1: each rotation is taken from the
 * previous one (the paper's "incremental rotations"). */
he_status he_conv2d(he_ctx *ctx, he_ct *const *in, uint32_t ch_in, const double *w, const double *bias,
                    uint32_t ch_out, uint32_t K, uint32_t S, int incremental, he_ct **out);
he_status he_conv1d(he_ctx *ctx, he_ct *const *in, uint32_t ch_in, const double *w, const double *bias,
                    uint32_t ch_out, uint32_t K, uint32_t S, int incremental, he_ct **out);
/* Sec. IV-C: c x c average pooling by rotations and additions, no level;
 * the factor 1/c^2 is carried in the layout and folded into the next linear layer. */
he_status he_avgpool(he_ctx *ctx, he_ct *const *in, uint32_t ch, uint32_t c, he_ct **out);
/* Sec. IV-E: remove intervals and invalid values and pack ch channels into one
 * ciphertext (values at slots [0, ch*W*H) of each sample). */
he_status he_flatten(he_ctx *ctx, he_ct *const *in, uint32_t ch, he_ct **out);
/* Algorithm 2: FC din -> dout on a flattened ciphertext; W [dout][din], b [dout]. */
he_status he_fc(he_ctx *ctx, const he_ct *in, const double *W, const double *b, uint32_t din,
                uint32_t dout, he_ct **out);

/* ---- compiled models, batched inference ------------------------------- */
enum { HE_CONV2D = 1, HE_CONV1D = 2, HE_SQUARE = 3, HE_AVGPOOL = 4, HE_FLATTEN = 5, HE_FC = 6, HE_APPROX_RELU = 7 };
typedef struct {
    uint32_t op;       /* HE_CONV2D ... HE_APPROX_RELU */
    uint32_t ch_in;    /* conv: input channels; FC: DAT_in */
    uint32_t ch_out;   /* conv: output channels; FC: DAT_out */
    uint32_t k;        /* conv kernel size; average-pooling size; FC: how the final rotation sum
                          sum_{i < W_vec/DAT_out} Rot(C, i*DAT_out) of Alg. 2 is evaluated --
                          0 as printed (one hoisted combination of the rotations), 1 by binary
                          doubling (about log2 + popcount rotations; other key switches, so other
                          ciphertexts, same slot values) */
    uint32_t stride;   /* conv stride */
    const double *w;   /* conv [ch_out][ch_in][k][k] (1-D: [ch_out][ch_in][k]); FC [ch_out][ch_in] */
    const double *b;   /* [ch_out] */
} he_layer;

/* Plan a layer list for W_img x H_img inputs (H_img = 1: 1-D): the slots a
 * sample needs (paper Sec. V), the levels consumed and the distinct rotation
 * steps (to pass to he_keygen).  steps may be NULL to query *n_steps. */
he_status he_model_plan(const he_layer *layers, size_t n, uint32_t W_img, uint32_t H_img,
                        uint32_t *stride, uint32_t *levels, int32_t *steps, size_t *n_steps);
/* he_model_plan for a given schedule (HE_SCHEDULE_*): the literal schedule never merges the
 * flatten's last stage with the channel packing, so its step set differs; he_model_plan is
 * this call with HE_SCHEDULE_FUSED. */
he_status he_model_plan_schedule(const he_layer *layers, size_t n, uint32_t W_img, uint32_t H_img,
                                 uint32_t schedule, uint32_t *stride, uint32_t *levels, int32_t *steps,
                                 size_t *n_steps);
/* Compile a layer list (paper Sec. IV: the model is fixed on the server side and its
 * layers are converted to HE operations once -- Algorithm 1 kernels, Algorithm 2's
 * pre-rotated weight matrix M_rot, the flatten masks of Sec. IV-E), for inputs of the
 * flattened layout with samples_per_ct samples per ciphertext (Sec. III-B).  Copies the
 * weights; the plaintext masks are encoded on the device at the first he_infer and
 * cached in the model.  Errors: HE_ENOKEY, HE_ELEVEL, HE_ESLOTS. */
he_status he_model_compile(he_ctx *ctx, const he_layer *layers, size_t n, uint32_t W_img, uint32_t H_img,
                           uint32_t samples_per_ct, he_model **out);
/* Run the compiled model on a ciphertext batch (paper Sec. III, Fig. 1: the server
 * evaluates the network on the client's ciphertexts; Sec. III-B: each ciphertext carries
 * samples_per_ct samples; Sec. IV-A: an input with more levels than the model consumes is
 * first reduced by Drop-Level).  All layers, every ciphertext of the batch in the same
 * kernel launches; *out receives the logits batch.
 * use_graph = 1 replays a captured CUDA graph after the first call of a given
 * batch size. */
he_status he_infer(he_model *m, const he_ct *in, int use_graph, he_ct **out);
/* Memory for the encoded weight masks of a convolution (0, the default: no limit, every
 * mask is encoded once and kept).  A convolution whose masks over Q u P take more than
 * `bytes` keeps only their sparse description on the device and encodes them at every
 * inference, in groups of output channels whose masks fit in `bytes` (more work per
 * inference, bounded memory; the results are bit-identical).  Takes effect for layers
 * not yet run.  Errors: HE_EINVAL. */
he_status he_model_set_mask_budget(he_model *m, uint64_t bytes);
void he_model_free(he_model *m);

/* ---- autotuning --------------------------------------------------------- */
/* Chooses the launch shapes of the batched path for this context's N, chain,
 * dnum and GPU by timing each candidate with CUDA events on scratch data (about
 * 4 GB at N = 2^14, released afterwards): limb split over 2-CTA clusters for the
 * NTT, ModDown and rescale kernels; outputs and polynomials per MAC launch; ciphertexts per
 * thread and grid order of the hoisted key-switch accumulation.  No choice
 * changes a result bit.  cache_path (optional) is a JSON file keyed by device
 * name and parameters: an entry there is used without measuring, a new
 * measurement is added to it.  report (optional) receives the timings as JSON.
 * Call it before he_model_compile / the first he_infer: captured CUDA graphs
 * keep the shapes they were captured with.  Errors: HE_EINVAL, HE_ENOMEM, HE_ECUDA. */
he_status he_autotune(he_ctx *ctx, const char *cache_path, char *report, size_t report_len);
/* The tuned knobs in the order: NTT limb layout, ModDown limb layout, rescale limb layout
 * (0 one CTA per limb, 1 a 2-CTA cluster, 2 two launches: outer stages over columns,
 * inner stages over 1024-coefficient blocks), MAC output group, key-switch ciphertexts
 * per thread, key-switch grid order, polynomials per MAC CTA, threads per coefficient of
 * a MAC group, ciphertexts per thread of the one-pass combination, the number of
 * ciphertexts from which a single-output weighted combination of one channel folds its
 * weights into the keys (default 16; not timed by he_autotune), the largest prime (in
 * bytes: 0 for none, the default; 5 for the 40-bit primes; 8 for every prime) whose limbs of
 * a mask MAC of six or more outputs run on the tensor cores (-1 = default).
 * he_tuning_set overrides them (values outside a knob's candidates fall back to the
 * nearest valid launch shape). */
he_status he_tuning_get(he_ctx *ctx, int32_t *values, size_t n);
he_status he_tuning_set(he_ctx *ctx, const int32_t *values, size_t n);

/* ---- serving ----------------------------------------------------------- */
/* A continuous-batching request loop over compiled models (the paper's
 * service model: clients send ciphertexts encrypted under their public key,
 * the server evaluates the network with the evaluation keys and returns
 * encrypted results; paper Sec. III).  One host thread serves every added
 * model, each from a FIFO queue: while a model has fewer than max_inflight
 * batches in flight, the queued requests (in arrival order, up to max_batch
 * ciphertexts) are gathered into one batch (padded to a power of two unless
 * exact_batches) and run on the model's stream; requests that arrive meanwhile
 * join the next batch.
 * A request's result is bit-identical whether it ran alone or in a mix.
 * Thread safety: submit / wait / stats may be called from any thread; the
 * contexts of the added models stay usable from other threads (every entry
 * point takes its context's lock). */
typedef struct he_server he_server;
typedef struct {
    uint32_t max_batch;     /* ciphertexts per launch of one model; rounded down to a power of two, >= 1 */
    uint32_t max_wait_us;   /* while a model's batch runs, a partial next batch waits up to this long for
                               more requests before it is launched behind it; 0: launch at once */
    uint64_t mem_budget;    /* device bytes for the models (their contexts' pools: keys and cached masks,
                               and their graph pools) plus the input ciphertexts of the requests
                               submitted and not yet collected (queued, running, or finished and
                               waiting for he_server_wait); 0: unlimited */
    uint32_t max_inflight;  /* batches of one model queued on its stream at once; 0: 2.  With 1, the
                               next batch is formed when the running one completes (larger batches
                               under load, one model's work never queued behind itself) */
    uint32_t exact_batches; /* 0: a batch is padded to a power of two (log2(max_batch)+1 graphs per
                               model); 1: one graph per batch size 1..max_batch, no padding.
                               Under load, max_inflight = 1 with exact_batches = 1 gave the lower
                               median and tail latency (bench.py --serve uses them) */
} he_server_opts;
typedef struct {
    uint64_t requests;        /* finished requests */
    uint64_t batches;         /* launched batches */
    uint64_t cts;             /* ciphertexts launched, padding included */
    double mean_batch;        /* cts / batches */
    double p50_ms, p99_ms, max_ms;   /* latency from submit to completion on the device (nearest rank) */
    uint64_t resident_bytes;  /* bytes the added models hold against the budget */
} he_server_stats;

/* Starts the loop's thread.  HE_EINVAL if max_batch is 0. */
he_status he_server_create(const he_server_opts *opt, he_server **out);
/* Adds a compiled model (borrowed: it must outlive the server).  Runs the model
 * once on zero ciphertexts for every batch shape (1, 2, 4, .. max_batch, or
 * 1, 2, 3, .. max_batch with exact_batches) at the
 * context's top level, capturing their CUDA graphs, then admits it: HE_ENOMEM
 * if the budget cannot hold what the model and its context keep on the device.
 * The ids are 0, 1, 2, ... in order of addition. */
he_status he_server_add_model(he_server *srv, he_model *model, uint32_t *model_id);
/* Queues a request: the ciphertext batch `in` (a fresh encryption of the
 * model's input layout, at most max_batch ciphertexts, on the model's context).
 * The server keeps its own reference to the buffer; the caller may free `in`.
 * HE_ENOMEM when admitting it would exceed the budget: the request is not
 * queued; it is admitted when submitted again after he_server_wait has
 * collected enough results (admission by memory, paper Sec. III service model:
 * the server holds every client's ciphertexts until they are returned).
 * HE_EINVAL / HE_ELEVEL when it does not fit the model. */
he_status he_server_submit(he_server *srv, uint32_t model_id, const he_ct *in, uint64_t *req_id);
/* Waits up to timeout_ms for a request and collects it: *out receives the
 * result (caller frees it with he_ct_free; NULL out frees it), *latency_ms
 * (optional) the time from submit to completion.  HE_ETIMEOUT leaves the
 * request pending; any other status ends it (the status of its batch). */
he_status he_server_wait(he_server *srv, uint64_t req_id, uint32_t timeout_ms, he_ct **out, double *latency_ms);
/* Non-blocking: *done = 1 once the request has finished (collect it with
 * he_server_wait), 0 while it is queued or running.  HE_EINVAL for an unknown
 * (or already collected) request. */
he_status he_server_poll(he_server *srv, uint64_t req_id, int *done);
/* Counters and latency percentiles of one model (model_id) or all (-1). */
he_status he_server_stats_get(he_server *srv, int32_t model_id, he_server_stats *out);
/* Runs every queued request to completion, frees uncollected results, stops the thread. */
void he_server_destroy(he_server *srv);
/* The same loop on simulated models, without a GPU: request k arrives at
 * arrival_us[k] (microseconds after the start, nondecreasing) for model
 * model_of[k] with cts_of[k] ciphertexts; a batch of b ciphertexts of model i
 * occupies one simulated device for base_us[i] + per_ct_us[i]*b microseconds
 * (batches back to back).  Outputs (optional): the batch id of each request
 * (ids increase in launch order) and its latency.  Runs in real time. */
he_status he_server_simulate(const he_server_opts *opt, uint32_t n_models, const double *base_us,
                             const double *per_ct_us, size_t n_req, const double *arrival_us,
                             const uint32_t *model_of, const uint32_t *cts_of, uint64_t *batch_of,
                             double *latency_ms);
/* he_server_simulate with memory admission: every simulated ciphertext counts as one
 * byte of opt->mem_budget (the simulated models hold none) from its request's
 * submission until the request completes.  A request the budget cannot hold on
 * arrival is refused (refusals[k] = 1, else 0) and submitted again, in arrival order
 * behind earlier refused ones, as completions free the budget; its latency counts
 * from its arrival.  refusals is optional. */
he_status he_server_simulate_admission(const he_server_opts *opt, uint32_t n_models, const double *base_us,
                                       const double *per_ct_us, size_t n_req, const double *arrival_us,
                                       const uint32_t *model_of, const uint32_t *cts_of, uint64_t *batch_of,
                                       double *latency_ms, uint32_t *refusals);

/* ---- low level ------------------------------------------------------- */
/* In-place forward (inverse = 0) or inverse negacyclic NTT of n_limbs device
 * limbs data[n_limbs][N]; limb i uses prime prime_idx[i] (index into the
 * chain of he_context_primes).  Forward output is bit-reversed evaluation order. */
he_status he_ntt(he_ctx *ctx, uint64_t *data, uint32_t n_limbs, const uint32_t *prime_idx, int inverse);
/* Rescale that allocates no device memory.  The paper has no counterpart: this
 * is a library service for callers that cannot allocate when they rescale --
 * code inside a CUDA stream capture (an allocation breaks the capture),
 * serving processes that reserve their whole memory budget up front and must
 * not fail with out-of-memory mid-request, and hosts whose device memory is
 * owned by another allocator.
 * in: device [batch][2][limbs][N] evaluation-form ciphertexts (the he_ct
 * layout); out: device [batch][2][limbs-1][N]; the result equals he_rescale's.
 * in and out must not overlap (the output's limb stride differs from the
 * input's, so an in-place call cannot work): overlapping ranges get HE_EINVAL.
 * Work is queued on the context's stream.  The only working memory is a
 * file-scope device array of 2^19 words (4 MiB) held by every GPU that loads
 * the library until the process exits: batch*2*N must not exceed 2^19 (16
 * ciphertexts at N = 2^14), else HE_EINVAL; N = 2^15 contexts get HE_EINVAL
 * (the kernels hold a whole limb in one CTA).  The array is fully overwritten
 * before use; calls share it, so calls that overlap on the GPU (other streams
 * or contexts on the same device) race.  The first call on a device looks up
 * the array's device address and sets kernel attributes: make that first call
 * before any stream capture.  Errors: HE_EINVAL, HE_ELEVEL (limbs < 2), HE_ECUDA. */
he_status he_rescale_noalloc(he_ctx *ctx, const uint64_t *in, uint64_t *out, uint32_t batch, uint32_t limbs);

/* Block until the context's stream is idle. */
he_status he_sync(he_ctx *ctx);
/* Number of kernels this context has launched so far (a graph replay counts
 * the kernels of the graph). */
uint64_t he_kernel_launches(const he_ctx *ctx);

/* Per-kernel timing: between he_profile_begin and he_profile_end every kernel
 * the context launches eagerly is bracketed by two CUDA events on the
 * context's stream.  he_profile_end synchronises and aggregates by kernel
 * name: launches, summed event time, and the algorithmic bytes of those
 * launches (the bytes the operation must read and write at least once). */
typedef struct {
    char name[32];
    uint64_t launches;
    double total_ms;
    double bytes;   /* algorithmic bytes */
    double ops;     /* algorithmic primitive operations: NTT butterflies (NTT, ModDown, rescale)
                       or 64x64->128 multiply-accumulates (MAC, key inner products) */
} he_kernel_stat;
/* Measured integer roofline: register-only throughput on this device of the
 * modular primitives the kernels use.  out[0] = lazy NTT butterflies/s,
 * out[1] = 64x64->128-bit multiply-accumulates/s, out[2] = Barrett modular
 * products/s, out[3] = the device's SM count (each kernel's grid is that many SMs
 * times the CTAs per SM it reaches).  out holds 4 doubles.  Runs a few short
 * kernels on the context's stream and waits. */
he_status he_ubench(he_ctx *ctx, double *out);

he_status he_profile_begin(he_ctx *ctx);
he_status he_profile_end(he_ctx *ctx, he_kernel_stat *out, size_t cap, size_t *n);

const char *he_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* UNIHENN_H */
