// Device-side tables and kernel launchers of the RNS-CKKS hot path.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "modarith.cuh"

#define FHE_MAX_LIMBS 64

// kernel launches issued so far by this library (all launchers count)
unsigned long long fhe_launch_counter();
// graph replays add the kernels they launch (captured launches are not run)
void fhe_launch_counter_add(long long n);

// One prime of the chain q_0..q_L, p_0..p_{alpha-1}.
struct PrimeTab {
    ModQ m;
    u64 n_inv, n_inv_sh;            // N^-1 mod q and its Shoup companion
    const ulonglong2 *fwd;          // [N] (psi^brv(k), Shoup)
    const ulonglong2 *inv;          // [N] (psi^-brv(k), Shoup)
};

// Per-level constants of hybrid key switching and rescale (device pointers).
struct LevelTab {
    int level, n_digits, ext;       // ext = level + 1 + alpha
    // iNTT epilogue of ModUp: N^-1 * (Qhat_{j,i})^-1 mod q_i, Shoup pair, [level+1]
    const ulonglong2 *y_scale;
    // (Qhat_{j,i} mod prime of ext limb t), [n_digits][alpha][ext]
    const u64 *modup_hat;
    // rescale by q_level: q_level^-1 mod q_i, Shoup pair, [level]
    const ulonglong2 *q_last_inv;
    // q_level mod q_i, [level]
    const u64 *q_last_mod;
};

// Context passed by value to kernels.
struct DevCtx {
    const PrimeTab *primes;         // [L+1+alpha]
    int logN, L, alpha;
    int logR1, logR2;               // NTT split: columns of 2^logR1, rows of 2^logR2
    // ModDown constants (level independent)
    const ulonglong2 *md_z_scale;   // [alpha] N^-1 * Phat_m^-1 mod p_m (Shoup)
    const u64 *md_z_add;            // [alpha] floor(P/2) * Phat_m^-1 mod p_m
    const u64 *md_phat;             // [alpha][L+1] Phat_m mod q_i
    const u64 *md_halfp;            // [L+1] floor(P/2) mod q_i
    const ulonglong2 *md_pinv;      // [L+1] P^-1 mod q_i (Shoup)
    // exact conversion from P: u = floor(sum_m z_m w_m / 2^md_E) counts the
    // multiples of P the fast conversion adds; w_m = floor(2^md_E / p_m)
    const u64 *md_w;                // [alpha]
    const u64 *md_pmod;             // [L+1] P mod q_i
    int md_E;                       // 63 + smallest bit length of the p_m
};

__host__ __device__ inline int ext_prime(int l, int level, int L) {
    // extended basis Q_level u P: limbs 0..level are q_0..q_level, then p_*
    return l <= level ? l : L + 1 + (l - level - 1);
}

// A set of limbs: item i, limb l at base + i*item + l*N (in words).
struct LimbSet {
    u64 *base;
    long long item;
    int n_items;
    int n_limbs;
};

// Rotation / relinearisation key switch of a batch of ciphertexts at one level.
struct KsArgs {
    const u64 *d;           // poly to switch, NTT domain: d + i*d_item, limbs 0..level
    long long d_item;
    int galois;             // Galois element applied to d (and to add0) on load; 1 = none
    const u64 *key;         // [n_digits_top][2][L+1+alpha][N]
    int key_digits_top;     // digits of the key at the top level
    const u64 *add0;        // addend of output poly 0 (nullable), limbs 0..level, + i*add_item
    const u64 *add1;        // addend of output poly 1 (nullable)
    long long add_item;
    int ip_galois;          // Galois gather applied to every limb entering the inner product (0/1: none)
    int ip_accumulate;      // inner product adds into the accumulator instead of overwriting it
    int add_galois;         // Galois gather of add0 in the output (0: same as galois)
    const u64 *base;        // added to both output polys without gather (nullable; may alias out)
    long long base_item;
    u64 *out;               // [item][2][level+1][N]
    long long out_item;
    int n_items;
    int level;
    // workspace (item-major): y [level+1], mu [digits][ext], acc [2][ext],
    // z [2][alpha], md [2][level+1], u [2] limbs; sized by the caller
    u64 *ws;
    long long ws_item;      // words per item
    // double hoisting (all nullable):
    u64 *ip_out;            // the inner product writes its [2][ext] result here (+ i*ip_out_item), not to ws
    long long ip_out_item;
    const u64 *ip_fold;     // with ip_out: poly 0 also gets (P mod q_t) sigma_ip_galois(ip_fold)[t], limbs t <= level
    long long ip_fold_item;
    const u64 *md_in;       // ModDown reads its [2][ext] input here (+ i*md_in_item), not ws's accumulator
    long long md_in_item;
};

size_t ks_workspace_words(const DevCtx &c, int level);
// Several baby-step rotations of one ModUp at once, each kept in Q_l u P
// (double hoisting).  Rotation k's inner product at output slot j reads the
// digits at sigma_k's source slot of j; here each thread takes two source
// slots, reads the digits and c0 there once for all rotations, and for
// rotation k reads its key at, and writes its result to, the output slots
// that those source slots feed (gal_inv[k]: the inverse Galois element).
// The products, sums and reductions are those of the one-rotation form.
#define KS_BABIES_MAX 8
struct IpBabies {
    int n;
    const u64 *key[KS_BABIES_MAX];
    u64 *out[KS_BABIES_MAX];
    int gal_inv[KS_BABIES_MAX];
};
// a: d (c1 of the input), ip_fold (its c0), ip_out_item, n_items, level, ws
// / ws_item holding the ModUp digits.  Up to 7 digits; else
// cudaErrorInvalidValue (the caller takes the one-rotation form).
cudaError_t launch_ks_ip_babies(const DevCtx &c, const LevelTab &lt, const KsArgs &a, const IpBabies &bb,
                                cudaStream_t s);
// ev (nullable): 9 events recorded on s before each of the 8 kernels and after the last.
// phases: KS_MODUP (inverse NTT, basis conversion, NTT), KS_IP (key inner
// product), KS_MODDOWN (back to Q, output); a plain key switch runs all three.
#define KS_MODUP 1
#define KS_IP 2
#define KS_MODDOWN 4
#define KS_ALL 7
cudaError_t launch_keyswitch(const DevCtx &c, const LevelTab &lt, const KsArgs &a, cudaStream_t s,
                             cudaEvent_t *ev = nullptr, int phases = KS_ALL);
// out[i][t] = (accumulate ? out[i][t] : 0) + sigma_galois(in[i][t]) for limbs t <= level (one poly)
cudaError_t launch_gather_acc(const DevCtx &c, const u64 *in, long long in_item, u64 *out, long long out_item,
                              int n_items, int level, int galois, int accumulate, cudaStream_t s);

// Rescale: out[i] = q_l^-1 (in[i] - [in[l]]_centred) mod q_i for i < level, both polys.
struct RescaleArgs {
    const u64 *in;
    long long in_item;      // item stride; poly stride is (level+1)*N
    u64 *out;
    long long out_item;     // poly stride is level*N
    int n_items;
    int n_poly;
    int level;              // input level (>= 1)
    u64 *ws;                // [n_items*n_poly][N]
};
cudaError_t launch_rescale(const DevCtx &c, const LevelTab &lt, const RescaleArgs &a, cudaStream_t s);

// Plain forward/inverse NTT of limbs; limb l of item i uses prime pidx[l].
struct NttArgs {
    const u64 *src;
    u64 *dst;
    long long src_item, dst_item;
    int n_items, n_limbs;
    unsigned char pidx[FHE_MAX_LIMBS];
};
cudaError_t launch_ntt(const DevCtx &c, const NttArgs &a, bool inverse, cudaStream_t s);

// Elementwise ops over ciphertext limbs (limb l uses prime l).
cudaError_t launch_add(const DevCtx &c, const u64 *a, long long a_item, const u64 *b, long long b_item,
                       u64 *out, long long out_item, int n_items, int n_poly, int level, int subtract,
                       cudaStream_t s);
// out[p][l] = a[p][l] * (const[l]) for every poly p
cudaError_t launch_mul_const(const DevCtx &c, const u64 *a, long long a_item, const u64 *cst,
                             u64 *out, long long out_item, int n_items, int n_poly, int level,
                             cudaStream_t s);
// out[0][l] = a[0][l] + cst[l] (constant polynomial), out[1] = a[1]
cudaError_t launch_add_const(const DevCtx &c, const u64 *a, long long a_item, const u64 *cst,
                             u64 *out, long long out_item, int n_items, int level, cudaStream_t s);
// Tensor square with the activation's lower terms folded in:
//   d0 = c0^2 + C1 c0 + C0, d1 = 2 c0 c1 + C1 c1, d2 = c1^2
// with C1, C0 either one residue per limb (c1[l], c0[l]; nullable) or, when
// c1v is non-null, NTT-domain plaintexts per ciphertext of the tensor: item
// i uses c1v / c0v + (i % n_ct) * (level+1) * N (per-channel coefficients).
cudaError_t launch_square_act(const DevCtx &c, const u64 *in, long long in_item, const u64 *c1,
                              const u64 *c0, u64 *out, long long out_item, int n_items, int level,
                              cudaStream_t s, const u64 *c1v = nullptr, const u64 *c0v = nullptr, int n_ct = 1);
// copy limbs 0..new_level of every poly (mod-drop)
cudaError_t launch_drop(const DevCtx &c, const u64 *in, long long in_item, int in_level, u64 *out,
                        long long out_item, int new_level, int n_items, int n_poly, cudaStream_t s);
// m = c0 + c1*s (NTT domain), limbs 0..level
cudaError_t launch_decrypt(const DevCtx &c, const u64 *ct, const u64 *s_ntt, u64 *m, int level,
                           cudaStream_t s);

// Plaintext-ciphertext multiply-accumulate of a linear layer.  Output group
// g (one accumulator ciphertext per image) is
//   out_g = sum_{t in terms(g)} pt_t (.) srcs[src_t]   (+ bias_g on poly 0)
// where a source is a ciphertext tensor (image i at base + i*item).  Terms
// that share a plaintext (clustered weights) may be given as a run: the
// run's sources are added mod q first and multiplied by the plaintext once
// (grouped accumulation; the same residues, fewer products).
struct MacSrc {
    const u64 *base;      // image 0's ciphertext (2 polys x limbs, limbs as MacArgs.ext says)
    long long item;       // per-image stride
};
struct MacTerm {
    int src;              // index into srcs
    int run;              // first term of a run: the run's length (terms that share pt, consecutive); else 0 or 1
    const u64 *pt;        // plaintext limbs x N (its first level+1 limbs are Q's when ext)
};
struct MacGroup {
    u64 *out;             // image 0's output ciphertext
    long long out_item;   // per-image stride of out
    const u64 *bias;      // plaintext added to poly 0 (nullable)
    int term_begin, term_end;
    int accumulate;       // add to the output's current value instead of overwriting it
};
struct MacArgs {
    const MacGroup *groups;   // device arrays
    const MacTerm *terms;
    const MacSrc *srcs;
    int n_groups;
    int n_items;
    int level;
    int n_srcs;               // entries of srcs
    int images_per_cta;       // 1, 2, 4, 8, or 0: the batch rounded up to 2^k, at most 8
    int ext;                  // 0: limbs 0..level of q_0..q_level; 1: the level+1+alpha limbs of Q_level u P
};
cudaError_t launch_mac(const DevCtx &c, const MacArgs &a, cudaStream_t s);

// Device copy of the slot encoder's tables (the host encoder's own values):
// FFT twiddles of the stage of length 2^s at re/im + off[s] (2^(s-1)
// entries), the twist cos / sin(pi k / N), and perm[j] = brv(slot_pos[j]),
// where slot j lands before the first butterfly stage.
struct EncTab {
    const double *fft_re, *fft_im;
    long long off[24];
    const double *tw_c, *tw_s;
    const unsigned *perm;
};
// On-demand encoding of V term vectors given sparsely (row vids[v] of
// begin/slot/val) at `scale`, into NTT-domain limbs 0..level at
// pt + v * (level+1) * N (ext: the level+1+alpha limbs of Q_level u P, at
// pt + v * (level+1+alpha) * N).  buf: V * N doubles of scratch.  The
// operations are the host encoder's in its order (no contraction), so the
// limbs equal a resident encoding of the same dense vector.
cudaError_t launch_encode_sparse(const DevCtx &c, const EncTab &e, int V, const int *vids, const long long *begin,
                                 const int *slot, const double *val, double scale, int level, double *buf, u64 *pt,
                                 cudaStream_t s, bool ext = false);

// ChaCha20-based samplers (the stream of one (seed, domain, id0, id1)).
// uniform residues written directly as NTT-domain limbs
cudaError_t launch_sample_uniform(const DevCtx &c, uint64_t seed, uint32_t domain, uint32_t id0,
                                  uint32_t id1_base, uint32_t id1_step, u64 *out, int n_limbs,
                                  const unsigned char *pidx, cudaStream_t s);
// small signed samples (ternary or CBD-21) as int64 coefficients
cudaError_t launch_sample_small(const DevCtx &c, uint64_t seed, uint32_t domain, uint32_t id0,
                                uint32_t id1, int kind, long long *out, cudaStream_t s);
// signed int64 coefficients -> residues for limbs with primes pidx[l]
cudaError_t launch_signed_to_limbs(const DevCtx &c, const long long *v, u64 *out, int n_limbs,
                                   const unsigned char *pidx, cudaStream_t s);
// out[l] = a[l] (.) b[l] (+ c[l]) mod pidx[l]; sub: out = c - a*b
cudaError_t launch_mul_limbs(const DevCtx &c, const u64 *a, const u64 *b, const u64 *add, int negate,
                             u64 *out, int n_limbs, const unsigned char *pidx, cudaStream_t s);
// out[l] += cst[l] * x[l] mod pidx[l]
cudaError_t launch_axpy_limbs(const DevCtx &c, const u64 *x, const u64 *cst, u64 *out, int n_limbs,
                              const unsigned char *pidx, cudaStream_t s);
// integral doubles (any magnitude) -> residues of limbs 0..n_limbs-1 (prime l)
// ext_level >= 0: limb l takes prime ext_prime(l, ext_level, L) (Q_ext_level u P)
cudaError_t launch_double_to_limbs(const DevCtx &c, const double *v, u64 *out, int n_limbs, cudaStream_t s,
                                   int ext_level = -1);
// NTT-domain automorphism of limbs (gather): out[j] = in[pi_k(j)]
cudaError_t launch_automorphism(const DevCtx &c, const u64 *in, u64 *out, int n_limbs, int galois,
                                cudaStream_t s);
