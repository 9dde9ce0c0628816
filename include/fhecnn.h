/*
 * fhecnn.h -- C ABI of the GB300 (sm_103a) library for homomorphic CNN
 * inference under leveled RNS-CKKS with no bootstrapping.
 *
 * The paper (arxiv 2509.22857) states the problem as non-interactive
 * inference (Sec. 2.1, threat model): the client holds the input and the
 * CKKS secret key, encrypts and sends only ciphertexts; the server holds a
 * CNN with plaintext parameters, evaluates it homomorphically under leveled
 * FHE and returns encrypted logits that only the client decrypts.  The entry
 * points below follow that split: client-side calls (keygen, encode,
 * encrypt, decrypt, decode) and server-side calls (model load, convolution,
 * quadratic activation, pooling/dense, rescale, rotation, batched inference).
 * The scheme is RNS-CKKS as in Sec. 2.2: R_Q = Z_Q[x]/(x^N+1), Q = q_0..q_L
 * held as 64-bit residue limbs, a special modulus P (alpha primes) for hybrid
 * key switching.
 *
 * Conventions for every function:
 *   - Return value: 0 (FHE_OK) on success, a negative FHE_E_* code on error;
 *     fhe_last_error() then returns a thread-local message.  On error no
 *     output handle is written and inputs are unchanged.
 *   - Handles (fhe_ctx, fhe_sk, fhe_evk, fhe_pt, fhe_ct, fhe_model) are
 *     opaque, created and owned by the library, released with their *_free /
 *     *_destroy call.  A handle belongs to the context that made it and must
 *     not outlive it.
 *   - Host arrays passed in are owned by the caller and only read during the
 *     call; host arrays passed out are written during the call only.
 *   - Ciphertexts, plaintexts and keys live in device memory of the
 *     context's GPU; they are in the NTT domain, limb-major
 *     ([poly][limb][N] 64-bit words).  Data leaves the device only through
 *     fhe_ct_export / fhe_decrypt + fhe_decode.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream are asynchronous with respect to
 *     the host unless stated otherwise; calls without one synchronise.
 *   - Not thread-safe per context: calls on one context must be serialised
 *     by the caller.
 */
#ifndef FHECNN_H
#define FHECNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FHE_OK 0
#define FHE_E_INVAL -1    /* bad argument, size or handle */
#define FHE_E_LEVEL -2    /* no level left, or level / scale mismatch */
#define FHE_E_NOKEY -3    /* evaluation key for a rotation step is missing */
#define FHE_E_OOM -4      /* device or host allocation failed */
#define FHE_E_CUDA -5     /* a CUDA call failed (message has the CUDA error) */
#define FHE_E_TIMEOUT -6  /* a bounded device wait expired */

typedef struct fhe_ctx fhe_ctx;
typedef struct fhe_sk fhe_sk;
typedef struct fhe_evk fhe_evk;
typedef struct fhe_pt fhe_pt;
typedef struct fhe_ct fhe_ct;
typedef struct fhe_model fhe_model;
typedef struct fhe_pipeline fhe_pipeline;
typedef struct fhe_server fhe_server;

/*
 * Parameters (Table 4 and the appendix on FHE parameters: ring degree N,
 * scale Delta, L rescale primes, output prime q_0, special modulus P).
 * Primes are = 1 mod 2N, chosen in descending order below 2^bits: first the
 * L primes q_1..q_L of q_bits, then q_0 of q0_bits, then the alpha special
 * primes of p_bits, each skipping primes already taken.  alpha is also the
 * number of consecutive primes per key-switching digit.
 * Or `primes` gives the chain explicitly (the appendix on FHE parameters
 * prints the paper's chains): L+1+alpha values, q_0..q_L then
 * p_0..p_{alpha-1}, each prime, = 1 mod 2N, distinct and of 20..58 bits;
 * the *_bits fields are then ignored.
 * Limits: 12 <= log_n <= 16; generated primes 31..58 bits; 1 <= alpha <= 8;
 * L + 1 + alpha <= 64; at most 2^(62 - b) digits ceil((L+1)/alpha) for the
 * largest prime's size b (the key inner product sums one 2b-bit product per
 * digit below Barrett's 2^(b+62) bound).
 */
typedef struct {
    int log_n;
    int L;
    int q_bits;
    int q0_bits;
    int p_bits;
    int alpha;
    double log_scale;   /* Delta = 2^log_scale */
    int device;         /* CUDA device ordinal */
    const uint64_t *primes;   /* explicit chain, or NULL */
} fhe_params;

const char *fhe_last_error(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts); a monotonic counter for launch accounting. */
uint64_t fhe_kernel_launches(void);

/* Context: builds the prime chain, NTT tables and key-switching constants on
 * the device.  fhe_ctx_destroy frees everything the context made.  It also
 * sets the device's default stream-ordered memory pool (this process's
 * CUDA context only) to keep its memory mapped across synchronisations:
 * step temporaries come from it, and the library hands unused pool memory
 * back when a plain allocation of its own is refused. */
int fhe_ctx_create(const fhe_params *params, fhe_ctx **out);
int fhe_ctx_destroy(fhe_ctx *ctx);
/* q_0..q_L then p_0..p_{alpha-1} into out[cap]; *n = count (test hook). */
int fhe_ctx_primes(const fhe_ctx *ctx, uint64_t *out, size_t cap, size_t *n);
/* Execution tuning of a context (no effect on results; the paper has no
 * counterpart): a linear step processes its input ciphertexts in chunks of
 * at most lin_chunk_srcs MAC sources (inputs plus their baby-step
 * rotations; >= 2, default 160), so that the rotated copies of a wide
 * HW-layout layer are made and consumed a chunk at a time.  Returns
 * FHE_E_INVAL for a value below 2. */
int fhe_ctx_set_linear_chunk(fhe_ctx *ctx, int lin_chunk_srcs);
/* Device scratch, in bytes, for the plaintexts of a linear step encoded on
 * demand (fhe_step_desc.sparse_vec_begin): each row takes N doubles of FFT
 * buffer plus its limbs, and a step runs its output groups in batches whose
 * distinct rows fit (at least one group per batch; default 4 GiB).
 * Bit-neutral. */
int fhe_ctx_set_encode_scratch(fhe_ctx *ctx, size_t bytes);
/* At most max_items items per launch of a whole key switch of a network
 * step (activations, rotate-and-sum), so that its workspace is sized for
 * max_items (0, the default: any number).  Pipelines size their per-segment
 * workspaces by it when they are created.  Bit-neutral. */
int fhe_ctx_set_keyswitch_batch(fhe_ctx *ctx, int max_items);
/* Images per block of the plaintext MAC (1, 2, 4 or 8; 0, the default: the
 * batch rounded up to a power of two, at most 8).  A block owns 512 /
 * images_per_cta coefficients of one limb for that many images, so the
 * plaintext coefficients it loads serve every image of the block.
 * Bit-neutral (the sums are exact mod q).  A pipeline keeps the value its
 * graphs were captured with.  FHE_E_INVAL for other values. */
int fhe_ctx_set_mac_images(fhe_ctx *ctx, int images_per_cta);
/* Host-side fault injection (no counterpart in the paper): after `after`
 * further device allocations through the context succeed, the next one is
 * refused with FHE_E_OOM, as cudaMalloc's own refusal would be, and the
 * injection turns itself off.  after < 0 turns it off at once.  The failing
 * call frees what it allocated and leaves the context usable. */
int fhe_ctx_inject_alloc_failure(fhe_ctx *ctx, int after);

/* ---------------------------------------------------------------- client */

/*
 * Key generation (client side, Sec. 2.1).  Secret key s is ternary.  The
 * evaluation keys hold the relinearisation key (s^2 -> s) and one Galois key
 * per distinct rotation step in rot_steps[n_steps] (slot rotation left by
 * the step; 5^step mod 2N).  All randomness is the RFC 8439 ChaCha20 stream
 * with key (seed mod 2^32, seed >> 32, domain, 0, 0, 0, 0, 0), nonce
 * (id0, id1, 0) and block counter 0, 1, ...: domain 1 the secret key
 * (coefficient k: word k, floor(3w / 2^32) - 1), domain 2 the uniform key
 * masks (id0 = key id: 0 relinearisation, else the Galois element;
 * id1 = 65536 * digit + limb; coefficient k: words 4k..4k+3 as a 128-bit
 * integer mod q, drawn directly in the NTT domain), domain 3 the key errors
 * (id1 = digit; centred binomial, popcount of the low 21 bits of word 2k
 * minus that of word 2k+1).
 */
int fhe_keygen(fhe_ctx *ctx, uint64_t seed, const int32_t *rot_steps, size_t n_steps, fhe_sk **sk,
               fhe_evk **evk);
int fhe_sk_free(fhe_sk *sk);
int fhe_evk_free(fhe_evk *evk);
/* Galois elements present in the key set (test hook): out[cap], *n = count. */
int fhe_evk_galois(const fhe_evk *evk, int32_t *out, size_t cap, size_t *n);
/* Key transport between client and server (Sec. 2.2: the server holds only
 * the public evaluation keys).  Layouts are those of fhe_sk_export and
 * fhe_evk_export: NTT domain, limb t reduced mod prime t (q_0..q_L, then
 * p_0..p_{alpha-1}).
 * fhe_sk_import: (L+1+alpha)*N words.
 * fhe_evk_import: n_keys host buffers of words_per_key =
 * dnum*2*(L+1+alpha)*N words each (dnum = ceil((L+1)/alpha)), keys[i] the
 * key of Galois element galois[i], galois 0 = the relinearisation key
 * (exactly one).  Galois elements are odd, in [3, 2N), and distinct.
 * Buffers are caller-owned and read during the call only.  FHE_E_INVAL for
 * a wrong size, element or count, or a residue not below its prime; nothing
 * is allocated then. */
int fhe_sk_import(fhe_ctx *ctx, const uint64_t *buf, size_t n_words, fhe_sk **out);
int fhe_evk_import(fhe_ctx *ctx, const int32_t *galois, size_t n_keys, const uint64_t *const *keys,
                   size_t words_per_key, fhe_evk **out);

/*
 * Encoding (Sec. 2.2): n <= N/2 complex slots (re[i], im[i]; im may be NULL
 * for real slots; missing slots are zero) -> round(scale * sigma^-1(z)) as a
 * plaintext at `level` (limbs q_0..q_level).
 */
int fhe_encode(fhe_ctx *ctx, const double *re, const double *im, size_t n, double scale, int level,
               fhe_pt **out);
int fhe_pt_free(fhe_pt *pt);
/* Secret-key encryption: c1 = a (uniform), c0 = -a*s + e + m; a is domain 4
 * of the stream keyed by `seed` (id1 = limb), e domain 5. */
int fhe_encrypt(fhe_ctx *ctx, const fhe_sk *sk, const fhe_pt *pt, uint64_t seed, fhe_ct **out);
/* m = c0 + c1*s, as a plaintext at the ciphertext's level and scale. */
int fhe_decrypt(fhe_ctx *ctx, const fhe_sk *sk, const fhe_ct *ct, fhe_pt **out);
/* Slots of a plaintext: re[n], im[n] (im may be NULL), n <= N/2. */
int fhe_decode(fhe_ctx *ctx, const fhe_pt *pt, double *re, double *im, size_t n);

/* --------------------------------------------------------- ciphertexts */

int fhe_ct_free(fhe_ct *ct);
int fhe_ct_info(const fhe_ct *ct, int *level, int *n_poly, double *scale);
/*
 * Canonical export: coefficient domain, residues in [0, q_i), layout
 * [poly][limb][N]; cap is the capacity of buf in words
 * (needs n_poly*(level+1)*N).  Synchronous.
 */
int fhe_ct_export(const fhe_ct *ct, uint64_t *buf, size_t cap, int *level, double *scale, int *n_poly);
/* Inverse of fhe_ct_export. */
int fhe_ct_import(fhe_ctx *ctx, const uint64_t *buf, int n_poly, int level, double scale, fhe_ct **out);

/* --------------------------------------------- homomorphic primitives */

/* Slot rotation left by `step` (Sec. 2.2): Galois automorphism 5^step then
 * hybrid key switching (ModUp, key inner product, ModDown) with the Galois
 * key.  FHE_E_NOKEY if the key set lacks the step. */
int fhe_rotate(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *in, int step, fhe_ct **out, void *stream);
/* Ciphertext square then relinearisation: (c0,c1)^2 = (c0^2, 2c0c1, c1^2),
 * key-switch c1^2 with the relinearisation key.  Scale is squared. */
int fhe_square(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *in, fhe_ct **out, void *stream);
/* Rescale (Sec. 2.2, Sec. 4.3): divide by the top prime q_level with
 * rounding, drop one level, scale /= q_level.  In place on the handle.
 * FHE_E_LEVEL at level 0. */
int fhe_rescale(fhe_ctx *ctx, fhe_ct *ct, void *stream);
/* out = a + b.  Both operands must have the same level and the same scale
 * (relative difference at most 1e-9), else FHE_E_LEVEL (Sec. 4.3: addends
 * are brought to one level and scale before they are added). */
int fhe_add(fhe_ctx *ctx, const fhe_ct *a, const fhe_ct *b, fhe_ct **out, void *stream);
/* out = a * pt (slot-wise), scale multiplies. */
int fhe_mul_plain(fhe_ctx *ctx, const fhe_ct *a, const fhe_pt *pt, fhe_ct **out, void *stream);

/* ------------------------------------------------------------- models */

/* Step kinds of a compiled model program (see fhe_model_desc). */
#define FHE_STEP_LINEAR 1   /* convolution / dense: sum of diagonals (BSGS) */
#define FHE_STEP_RESCALE 2  /* rescale every ciphertext of a tensor */
#define FHE_STEP_ACT 3      /* x^2 + c1 x + c0 with relinearisation */
#define FHE_STEP_ROTSUM 4   /* x <- x + rot(x, s) for each step s (pooling) */
#define FHE_STEP_CMUL 5     /* multiply by an integer constant (shortcut) */
#define FHE_STEP_DROP 6     /* mod-drop to a lower level */
#define FHE_STEP_ADD 7      /* residual add of two tensors */

/*
 * One step of a compiled network (Sec. 5.1 slot layouts, Sec. 4.3 rescale
 * placement).  Tensors are numbered lists of ciphertexts (one per image).
 * LINEAR: for each output ciphertext o and giant step g,
 *     acc_{o,g} = sum_terms pt_term (.) rot(in[term_ct], term_baby)
 *     out_o     = bias_o + sum_g rot(acc_{o,g}, g)
 *   The baby-step rotations of one input share one ModUp (the Galois
 *   automorphism is applied to the extended limbs), and the giant-step
 *   rotations of one output share one ModDown (their inner products are summed
 *   in the extended basis Q_l u P first).
 *   where the term vectors (rows of vecs, n_slots doubles each; terms that
 *   share a row share one plaintext in HBM, as clustered weights do,
 *   Sec. 5.2) are encoded at w_scale and the bias vectors at bias_scale,
 *   both at the input's level.
 * ACT: c1 and c0 are integers (given as integral doubles of any size) that
 *   are already scaled: out = x^2 + c1*x + c0 (c0 added to poly 0).
 * CMUL: out = value * x (value an integral double).
 * ROTSUM: steps[n_steps] applied in order.
 * DROP: out = x restricted to limbs 0..level.
 * ADD: out = src + src2.
 */
typedef struct {
    int kind;
    int src, src2, dst;
    /* LINEAR */
    double w_scale, bias_scale;
    int n_groups;                    /* (out ct, giant step) groups */
    const int32_t *group_out;        /* [n_groups] */
    const int32_t *group_giant;      /* [n_groups] rotation step g (0 = none) */
    const int32_t *group_term_begin; /* [n_groups + 1] */
    const int32_t *term_ct;          /* [n_terms] input ciphertext index */
    const int32_t *term_baby;        /* [n_terms] baby rotation step b */
    const int32_t *term_vec_id;      /* [n_terms] row of vecs */
    int n_vecs;                      /* distinct term vectors (one plaintext each) */
    const double *vecs;              /* [n_vecs][n_slots] */
    int n_bias;
    const int32_t *bias_out;         /* [n_bias] output ciphertext index */
    const double *bias_vec;          /* [n_bias][n_slots] */
    /* ACT, CMUL */
    double c1, c0, value;
    /* ROTSUM */
    int n_steps;
    const int32_t *steps;
    /* DROP */
    int level;
    /*
     * LINEAR, encoded on demand (the paper's "Standard" evaluation, Sec. 5.2
     * and its appendix tables, where plaintext encoding is part of the
     * layer's cost): when sparse_vec_begin is non-null, vecs is unused and
     * row v of the term vectors is given by its nonzero entries
     * sparse_slot / sparse_val[sparse_vec_begin[v] .. sparse_vec_begin[v+1])
     * (slots < n_slots).  Nothing of these rows is encoded at load: each
     * time the step runs, the library encodes the plaintexts of a batch of
     * output groups on the device (the host encoder's operations in its
     * order, so the plaintexts are bit-identical to a resident encoding),
     * multiplies, and reuses the buffer for the next batch.  For layers
     * whose encoded plaintexts would not fit in device memory.
     */
    const int64_t *sparse_vec_begin; /* [n_vecs + 1] */
    const int32_t *sparse_slot;      /* [nnz] */
    const double *sparse_val;        /* [nnz] */
    /*
     * ACT with one coefficient pair per channel (node fusing Case 1, Sec. 4.1:
     * a batch norm fused into the activation): when act_c1_vecs is non-null,
     * c1 and c0 are unused and ciphertext k of the tensor computes
     * x^2 + v1_k (.) x + v0_k, with v1_k = act_c1_vecs[k] encoded at
     * act_c1_scale and v0_k = act_c0_vecs[k] at act_c0_scale (slot vectors,
     * [n_ct][n_slots]; encoded once at load, at the tensor's level).
     */
    const double *act_c1_vecs;
    const double *act_c0_vecs;
    double act_c1_scale, act_c0_scale;
    /*
     * LINEAR, double hoisting (hybrid key switching, Sec. 2: the special
     * modulus P of ModUp / ModDown).  0: every baby-step rotation is brought
     * back to Q_l by its own ModDown before the plaintext products.  1: the
     * baby-step rotations stay in the extended basis Q_l u P (the inner
     * product with the key plus P times the rotated c0), the terms with a
     * baby rotation are multiplied by plaintexts encoded over Q_l u P and
     * summed there, and each output group (out, giant step) takes one
     * ModDown, added to the group's unrotated terms (plain products over
     * Q_l) and bias.  The two differ only in the rounding of the ModDowns:
     * a different, equally valid ciphertext of the same values.
     */
    int double_hoist;
} fhe_step_desc;

typedef struct {
    int n_tensors;
    const int32_t *tensor_n_ct;      /* [n_tensors] ciphertexts per image */
    const int32_t *tensor_level;     /* [n_tensors] */
    const double *tensor_scale;      /* [n_tensors] */
    int input_tensor, output_tensor;
    int n_steps;
    const fhe_step_desc *steps;
} fhe_model_desc;

/* Encode every plaintext of the program at its level (weights stay
 * resident in HBM) and keep the program.  The description is copied. */
int fhe_model_load(fhe_ctx *ctx, const fhe_model_desc *desc, fhe_model **out);
int fhe_model_free(fhe_model *model);

/*
 * Per-step evaluation of one image.  `step` is the index of a LINEAR step
 * (fhe_eval_conv: convolutions), an ACT step (fhe_eval_quad_act, in place
 * on io[n]), or a ROTSUM / LINEAR step (fhe_eval_pool_dense: average pool
 * as a sum of rotations, dense layer as diagonals).  in[n_in] are the
 * step's input ciphertexts, out[n_out] receive new handles.
 */
int fhe_eval_conv(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, int step,
                  const fhe_ct *const *in, size_t n_in, fhe_ct **out, size_t n_out, void *stream);
int fhe_eval_quad_act(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, int step, fhe_ct **io,
                      size_t n, void *stream);
int fhe_eval_pool_dense(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, int step,
                        const fhe_ct *const *in, size_t n_in, fhe_ct **out, size_t n_out, void *stream);

/*
 * Whole-network inference of n_img images in one batched pass: in holds
 * n_img * n_in_ct input ciphertexts (image-major), out receives
 * n_img * n_out_ct handles.  Every kernel processes all images of a step
 * together, so evaluation keys and weight plaintexts are read once per batch.
 */
int fhe_infer(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, const fhe_ct *const *in,
              size_t n_img, fhe_ct **out, void *stream);

/*
 * fhe_infer with a timing breakdown: CUDA events on `stream` around every
 * phase; ms_by_kind[16] receives the summed milliseconds per phase kind:
 * [FHE_STEP_RESCALE], [FHE_STEP_ACT], [FHE_STEP_ROTSUM], [FHE_STEP_CMUL],
 * [FHE_STEP_DROP], [FHE_STEP_ADD], and for linear steps [10] baby-step
 * rotations, [11] plaintext MAC, [12] giant-step rotations.
 */
int fhe_infer_profiled(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, const fhe_ct *const *in,
                       size_t n_img, fhe_ct **out, void *stream, double *ms_by_kind);

/*
 * Continuous batching with images at mixed levels.  The program is cut after
 * every activation (and its rescale) into S segments; a group of up to
 * `group` images enters per tick and leaves S-1 ticks later, so up to
 * S*group images at S different levels are in flight at once.  All segments
 * of a tick run concurrently (one stream each); with use_graphs, each tick's
 * launches are captured into a CUDA graph (one per buffer parity, from the
 * third tick on) and replayed.  Evaluation keys and weight plaintexts are
 * shared by all groups.  Results are bit-identical to fhe_infer.
 */
int fhe_pipeline_create(fhe_ctx *ctx, const fhe_model *model, const fhe_evk *evk, int group, int use_graphs,
                        fhe_pipeline **out);
int fhe_pipeline_info(const fhe_pipeline *pipe, int *n_segments, int *group, int *n_in_ct, int *n_out_ct);
/*
 * One tick: in holds n_in (<= group) images' input ciphertexts (image-major,
 * n_in_ct each; n_in may be 0).  out (capacity group * n_out_ct) receives the
 * output ciphertexts of the group that leaves this tick, *n_out its image
 * count (0 while the pipeline fills) and *out_tag the tick at which that
 * group entered (-1 if none).  Synchronous.  The tick at which this call's
 * images enter is the value fhe_pipeline_ticks reports before the call.
 * Errors: a refusal found before launch (bad arguments, FHE_E_OOM for the
 * output ciphertexts) changes nothing: no image enters, the tick is not
 * counted, and the group due to leave leaves at the next call.  A failure
 * after launch (FHE_E_CUDA) still counts the tick and enters the images;
 * *n_out is then 0 and *out_tag names the group whose outputs were lost.
 */
int fhe_pipeline_tick(fhe_pipeline *pipe, const fhe_ct *const *in, size_t n_in, fhe_ct **out, size_t *n_out,
                      int64_t *out_tag);
/* Ticks counted so far (the entry tick of the next admitted group). */
int fhe_pipeline_ticks(const fhe_pipeline *pipe, int64_t *ticks);
int fhe_pipeline_free(fhe_pipeline *pipe);

/*
 * Serving (continuous batching): one server per context and key set.  Each
 * added model gets its own pipeline (above) and worker thread; requests are
 * queued per model and admitted into the next tick of their model's pipeline
 * while earlier requests are still inside it, and the workers of different
 * models tick concurrently.  fhe_server_add_model admits a model only if
 * cudaMemGetInfo reports at least reserve_bytes free (0: no check; the call
 * first synchronises the device and returns the stream-ordered pool's
 * unused memory to it) and its pipeline can be allocated (else FHE_E_OOM).
 * Weight plaintexts and evaluation keys stay resident.
 * fhe_server_submit takes ownership of the model's n_in_ct input ciphertexts
 * of one image (they are freed once admitted) and returns a ticket.
 * fhe_server_poll returns the request's n_out_ct output ciphertexts (new
 * handles owned by the caller) once done, and its latency from submit to
 * completion; *n_out = 0 while it is not done.  timeout_ms = 0 returns at
 * once, < 0 waits until done, > 0 waits at most that long and then returns
 * FHE_E_TIMEOUT (the request stays queued and can be polled again).
 * fhe_server_pause(server, 1) stops every worker before its next tick (a
 * stalled host worker: queued and in-flight requests wait, nothing is lost);
 * fhe_server_pause(server, 0) resumes them where they stopped.
 * fhe_server_stats: completed requests and the p50 / p99 of their latency.
 */
int fhe_server_create(fhe_ctx *ctx, const fhe_evk *evk, fhe_server **out);
int fhe_server_add_model(fhe_server *server, const fhe_model *model, int group, size_t reserve_bytes,
                         int *model_id);
int fhe_server_submit(fhe_server *server, int model_id, fhe_ct *const *in, uint64_t *ticket);
int fhe_server_poll(fhe_server *server, uint64_t ticket, int timeout_ms, fhe_ct **out, size_t cap, size_t *n_out,
                    double *latency_ms);
int fhe_server_pause(fhe_server *server, int paused);
int fhe_server_stats(fhe_server *server, uint64_t *completed, double *p50_ms, double *p99_ms);
int fhe_server_destroy(fhe_server *server);

/* ------------------------------------------------------ test hooks */

/* Forward (inverse = 0) or inverse NTT of n_limbs device limbs in place;
 * limb l uses prime index prime_idx[l] (0..L = q_i, L+1.. = p_j). */
int fhe_ntt_device(fhe_ctx *ctx, uint64_t *d_limbs, size_t n_limbs, const int32_t *prime_idx, int inverse,
                   void *stream);
/* Copy of one key-switching key (relinearisation: galois = 0) to host:
 * [digits][2][L+1+alpha][N] words, NTT domain. */
int fhe_evk_export(const fhe_evk *evk, int galois, uint64_t *buf, size_t cap, size_t *n_words);
/*
 * Timing hook: `iters` hybrid key switches (relinearisation key) of n_items
 * pseudo-random polynomials at `level`, after one warm-up, on `stream`, with
 * CUDA events recorded on that stream around each kernel of the pipeline.
 * ms_out[8] receives the mean duration of each kernel: ModUp inverse NTT
 * rows, inverse NTT columns (times Qhat^-1), basis conversion + NTT columns,
 * NTT rows + key inner product, ModDown inverse NTT rows, inverse NTT
 * columns, basis conversion + NTT columns, NTT rows + P^-1 output.
 * Synchronises with the stream.
 */
int fhe_profile_keyswitch(fhe_ctx *ctx, const fhe_evk *evk, int level, int n_items, int iters, float *ms_out,
                          void *stream);
/*
 * Rescale that allocates nothing (the paper has no counterpart: this is for
 * callers that cannot let the library call cudaMalloc -- their device memory
 * belongs to their own pool or to a fixed budget, or they cannot afford the
 * synchronisation an allocation brings).  Same result as fhe_rescale: in is
 * one ciphertext's [n_poly][level+1][N] NTT-domain limbs in device memory,
 * out receives [n_poly][level][N]; both are caller-owned and must not
 * overlap; the scale bookkeeping (scale / q_level) is the caller's.  The
 * scratch is a fixed 1 MiB device array inside the library (n_poly * N <=
 * 131072 words, i.e. two polynomials at N = 2^16), held by every GPU that
 * loads the library until the process exits; larger sizes are rejected with
 * FHE_E_INVAL.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress): make it before any stream capture.  That
 * address is kept for the life of the device's primary context: after
 * cudaDeviceReset (or anything else that destroys that context) do not call
 * this entry point again in the same process.  All
 * calls share the array, so calls that overlap on the GPU (other streams,
 * other threads) race; serialise them.  Asynchronous on `stream`.
 */
int fhe_rescale_noalloc(fhe_ctx *ctx, const uint64_t *in, uint64_t *out, int n_poly, int level, void *stream);
/* Secret key (NTT domain, all L+1+alpha limbs) to host. */
int fhe_sk_export(const fhe_sk *sk, uint64_t *buf, size_t cap);
/* Integer coefficients of an encoding, before reduction (host encoder),
 * as integral doubles: out[N]. */
int fhe_encode_coeffs(fhe_ctx *ctx, const double *re, const double *im, size_t n, double scale, double *out);

#ifdef __cplusplus
}
#endif
#endif
