/*
 * Plain CPU reference for the integer and encoding steps of leveled RNS-CKKS
 * (test infrastructure only: the product path never links or calls this file).
 *
 * Every routine here is the slow, direct form of the operation, written so a
 * reader can check it against its definition by eye:
 *   - modular products use a 128-bit product and the C '%' operator;
 *   - the NTT is the textbook iterative Cooley-Tukey / Gentleman-Sande pair and
 *     ntt_naive() is the O(N^2) evaluation it must equal;
 *   - base conversion is the fast (approximate) RNS basis extension written as
 *     its defining sum;
 *   - ChaCha20 is the RFC 8439 block function.
 * Paper sections followed: Sec. 2.2 (RNS-CKKS over R_Q = Z_Q[x]/(x^N+1) with Q
 * a product of primes and native 64-bit residues; encoding scales by Delta and
 * rounds; rotations; rescale; special modulus P for hybrid key switching).
 * Compiled with -ffp-contract=off so that the encoder's floating-point
 * operations happen in exactly the order written.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- modular */

uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}

uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = orc_mulmod(r, a, q);
        a = orc_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse by Fermat (q prime) */
uint64_t orc_invmod(uint64_t a, uint64_t q) {
    return orc_powmod(a, q - 2, q);
}

/* Deterministic Miller-Rabin for all 64-bit n (first twelve prime bases). */
int orc_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n % bases[i] == 0) return n == bases[i];
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = orc_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; r++) {
            x = orc_mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/*
 * Primes q = 1 (mod 2N) below 2^bits, taken in descending order: the
 * candidates are 2^bits - k*2N + 1 for k = 1, 2, ...  Primes listed in
 * `exclude` are skipped.  Returns the number written (count, or fewer if the
 * range runs out).
 */
int orc_gen_primes(int bits, int count, uint64_t two_n,
                   const uint64_t *exclude, int n_exclude, uint64_t *out) {
    int found = 0;
    uint64_t top = (uint64_t)1 << bits;
    for (uint64_t k = 1; found < count; k++) {
        if (k * two_n >= top) break;
        uint64_t c = top - k * two_n + 1;
        if (!orc_is_prime(c)) continue;
        int skip = 0;
        for (int i = 0; i < n_exclude; i++) if (exclude[i] == c) skip = 1;
        for (int i = 0; i < found; i++) if (out[i] == c) skip = 1;
        if (skip) continue;
        out[found++] = c;
    }
    return found;
}

/*
 * A primitive 2N-th root of unity mod q: psi = g^((q-1)/2N) for the smallest
 * g >= 2 that is a quadratic non-residue (g^((q-1)/2) = -1).  Then
 * psi^N = g^((q-1)/2) = -1, so psi has order exactly 2N.
 */
uint64_t orc_root_2n(uint64_t q, uint64_t two_n) {
    for (uint64_t g = 2;; g++) {
        if (orc_powmod(g, (q - 1) / 2, q) == q - 1)
            return orc_powmod(g, (q - 1) / two_n, q);
    }
}

static uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ---------------------------------------------------------------- NTT */

/*
 * Definition of the transform used everywhere in this project:
 *     A[j] = sum_i a[i] * psi^((2*brv(j)+1)*i)  mod q,   j = 0..N-1,
 * i.e. the evaluations of a(x) at the odd powers of psi (the roots of
 * x^N + 1), stored in bit-reversed order.  ntt_naive() computes exactly this
 * sum; ntt() computes it with the iterative Cooley-Tukey network.
 */
void orc_ntt_naive(const uint64_t *a, uint64_t *out, int logn, uint64_t q, uint64_t psi) {
    size_t n = (size_t)1 << logn;
    for (size_t j = 0; j < n; j++) {
        uint64_t e = 2 * (uint64_t)bitrev((uint32_t)j, logn) + 1;
        uint64_t root = orc_powmod(psi, e, q);
        uint64_t acc = 0, p = 1;
        for (size_t i = 0; i < n; i++) {
            acc = (acc + orc_mulmod(a[i], p, q)) % q;
            p = orc_mulmod(p, root, q);
        }
        out[j] = acc;
    }
}

void orc_ntt(uint64_t *a, int logn, uint64_t q, uint64_t psi) {
    size_t n = (size_t)1 << logn;
    uint64_t *tw = (uint64_t *)malloc(n * sizeof(uint64_t));
    for (size_t k = 0; k < n; k++) tw[k] = orc_powmod(psi, bitrev((uint32_t)k, logn), q);
    size_t t = n;
    for (size_t m = 1; m < n; m <<= 1) {
        t >>= 1;
        for (size_t i = 0; i < m; i++) {
            uint64_t w = tw[m + i];
            size_t j1 = 2 * i * t;
            for (size_t j = j1; j < j1 + t; j++) {
                uint64_t u = a[j];
                uint64_t v = orc_mulmod(a[j + t], w, q);
                a[j] = (u + v) % q;
                a[j + t] = (u + q - v) % q;
            }
        }
    }
    free(tw);
}

/* Inverse of orc_ntt: Gentleman-Sande with psi^-1, then a factor N^-1. */
void orc_intt(uint64_t *a, int logn, uint64_t q, uint64_t psi) {
    size_t n = (size_t)1 << logn;
    uint64_t psi_inv = orc_invmod(psi, q);
    uint64_t *tw = (uint64_t *)malloc(n * sizeof(uint64_t));
    for (size_t k = 0; k < n; k++) tw[k] = orc_powmod(psi_inv, bitrev((uint32_t)k, logn), q);
    size_t t = 1;
    for (size_t m = n >> 1; m >= 1; m >>= 1) {
        for (size_t i = 0; i < m; i++) {
            uint64_t w = tw[m + i];
            size_t j1 = 2 * i * t;
            for (size_t j = j1; j < j1 + t; j++) {
                uint64_t u = a[j];
                uint64_t v = a[j + t];
                a[j] = (u + v) % q;
                a[j + t] = orc_mulmod((u + q - v) % q, w, q);
            }
        }
        t <<= 1;
    }
    uint64_t n_inv = orc_invmod((uint64_t)n % q, q);
    for (size_t j = 0; j < n; j++) a[j] = orc_mulmod(a[j], n_inv, q);
    free(tw);
}

/* Negacyclic product by the schoolbook O(N^2) sum: x^N = -1. */
void orc_negacyclic_naive(const uint64_t *a, const uint64_t *b, uint64_t *out,
                          int logn, uint64_t q) {
    size_t n = (size_t)1 << logn;
    for (size_t k = 0; k < n; k++) out[k] = 0;
    for (size_t i = 0; i < n; i++) {
        for (size_t j = 0; j < n; j++) {
            uint64_t p = orc_mulmod(a[i], b[j], q);
            size_t k = i + j;
            if (k < n) out[k] = (out[k] + p) % q;
            else out[k - n] = (out[k - n] + q - p) % q;
        }
    }
}

/* ------------------------------------------------------ elementwise ops */

void orc_vec_add(const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = (a[i] + b[i]) % q;
}
void orc_vec_sub(const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = (a[i] + q - b[i]) % q;
}
void orc_vec_neg(const uint64_t *a, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = (q - a[i]) % q;
}
void orc_vec_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = orc_mulmod(a[i], b[i], q);
}
void orc_vec_mul_scalar(const uint64_t *a, uint64_t c, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = orc_mulmod(a[i], c, q);
}
void orc_vec_add_scalar(const uint64_t *a, uint64_t c, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) out[i] = (a[i] + c % q) % q;
}
/* signed integers -> residues mod q */
void orc_vec_from_signed(const int64_t *a, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) {
        int64_t v = a[i];
        if (v >= 0) out[i] = (uint64_t)v % q;
        else out[i] = (q - ((uint64_t)(-(v + 1)) + 1) % q) % q;
    }
}

/* integral doubles (any magnitude) -> residues mod q, exactly: below 2^63 via
 * int64, above as mantissa * 2^shift with a 53-bit integer mantissa */
void orc_vec_from_double(const double *a, uint64_t *out, size_t n, uint64_t q) {
    for (size_t i = 0; i < n; i++) {
        double v = a[i];
        double av = fabs(v);
        uint64_t r;
        if (av < 9223372036854775808.0) {
            r = (uint64_t)(int64_t)av % q;
        } else {
            int e;
            double mant = frexp(av, &e);
            uint64_t m = (uint64_t)ldexp(mant, 53);
            r = orc_mulmod(m % q, orc_powmod(2, (uint64_t)(e - 53), q), q);
        }
        out[i] = (v < 0) ? (q - r) % q : r;
    }
}

/*
 * Fast RNS basis conversion from the basis {q_in[0..n_in)} to a prime t:
 *     out[k] = sum_i [ x_i[k] * (Qin/q_i)^-1 ]_{q_i} * (Qin/q_i mod t)   mod t
 * where Qin is the product of the input primes.  This is the approximate
 * conversion: it returns x + u*Qin mod t for some 0 <= u < n_in.
 * `in` holds n_in limbs of length n (limb-major); one call per target prime.
 */
void orc_basis_convert(const uint64_t *in, const uint64_t *q_in, int n_in,
                       uint64_t t, uint64_t *out, size_t n) {
    uint64_t *hat_inv = (uint64_t *)malloc(n_in * sizeof(uint64_t));
    uint64_t *hat_t = (uint64_t *)malloc(n_in * sizeof(uint64_t));
    for (int i = 0; i < n_in; i++) {
        uint64_t h = 1, ht = 1 % t;
        for (int k = 0; k < n_in; k++) {
            if (k == i) continue;
            h = orc_mulmod(h, q_in[k] % q_in[i], q_in[i]);
            ht = orc_mulmod(ht, q_in[k] % t, t);
        }
        hat_inv[i] = orc_invmod(h, q_in[i]);
        hat_t[i] = ht;
    }
    for (size_t k = 0; k < n; k++) {
        uint64_t acc = 0;
        for (int i = 0; i < n_in; i++) {
            uint64_t y = orc_mulmod(in[(size_t)i * n + k], hat_inv[i], q_in[i]);
            acc = (acc + orc_mulmod(y % t, hat_t[i], t)) % t;
        }
        out[k] = acc;
    }
    free(hat_inv);
    free(hat_t);
}

/*
 * Overflow of the fast conversion above: with y_i = [x_i (Qin/q_i)^-1]_{q_i}
 * the sum  sum_i y_i (Qin/q_i)  equals x + u Qin for the x in [0, Qin) whose
 * residues are x_i, and u = floor(sum_i y_i / q_i) < n_in.  u is found here
 * exactly: the sum is formed as a multi-word integer and Qin is subtracted
 * while it is not below Qin.  (Words are little-endian 64-bit.)
 */
static void mp_mul_word(const uint64_t *a, int w, uint64_t b, uint64_t *out) {
    u128 carry = 0;
    for (int k = 0; k < w; k++) {
        u128 t = (u128)a[k] * b + carry;
        out[k] = (uint64_t)t;
        carry = t >> 64;
    }
}

static void mp_add(uint64_t *a, const uint64_t *b, int w) {
    u128 carry = 0;
    for (int k = 0; k < w; k++) {
        u128 t = (u128)a[k] + b[k] + carry;
        a[k] = (uint64_t)t;
        carry = t >> 64;
    }
}

static int mp_cmp(const uint64_t *a, const uint64_t *b, int w) {
    for (int k = w - 1; k >= 0; k--) {
        if (a[k] != b[k]) return a[k] > b[k] ? 1 : -1;
    }
    return 0;
}

static void mp_sub(uint64_t *a, const uint64_t *b, int w) {
    uint64_t borrow = 0;
    for (int k = 0; k < w; k++) {
        uint64_t bk = b[k] + borrow;
        uint64_t nb = (bk < borrow) || (a[k] < bk);
        a[k] -= bk;
        borrow = nb;
    }
}

void orc_conv_overflow(const uint64_t *in, const uint64_t *q_in, int n_in, uint64_t *u_out, size_t n) {
    const int w = n_in + 1;
    uint64_t *qhat = (uint64_t *)calloc((size_t)n_in * w, sizeof(uint64_t));
    uint64_t *qall = (uint64_t *)calloc(w, sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)calloc(w, sizeof(uint64_t));
    uint64_t *acc = (uint64_t *)calloc(w, sizeof(uint64_t));
    uint64_t *hat_inv = (uint64_t *)malloc(n_in * sizeof(uint64_t));
    qall[0] = 1;
    for (int i = 0; i < n_in; i++) {
        mp_mul_word(qall, w, q_in[i], tmp);
        memcpy(qall, tmp, w * sizeof(uint64_t));
        uint64_t *h = qhat + (size_t)i * w;
        h[0] = 1;
        uint64_t hm = 1;
        for (int k = 0; k < n_in; k++) {
            if (k == i) continue;
            mp_mul_word(h, w, q_in[k], tmp);
            memcpy(h, tmp, w * sizeof(uint64_t));
            hm = orc_mulmod(hm, q_in[k] % q_in[i], q_in[i]);
        }
        hat_inv[i] = orc_invmod(hm, q_in[i]);
    }
    for (size_t k = 0; k < n; k++) {
        memset(acc, 0, w * sizeof(uint64_t));
        for (int i = 0; i < n_in; i++) {
            uint64_t y = orc_mulmod(in[(size_t)i * n + k], hat_inv[i], q_in[i]);
            mp_mul_word(qhat + (size_t)i * w, w, y, tmp);
            mp_add(acc, tmp, w);
        }
        uint64_t u = 0;
        while (mp_cmp(acc, qall, w) >= 0) {
            mp_sub(acc, qall, w);
            u++;
        }
        u_out[k] = u;
    }
    free(qhat);
    free(qall);
    free(tmp);
    free(acc);
    free(hat_inv);
}

/* --------------------------------------------------------------- ChaCha20 */

static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

#define QR(a, b, c, d)                 \
    a += b; d ^= a; d = rotl32(d, 16); \
    c += d; b ^= c; b = rotl32(b, 12); \
    a += b; d ^= a; d = rotl32(d, 8);  \
    c += d; b ^= c; b = rotl32(b, 7);

/* RFC 8439 Sec. 2.3 block function: 20 rounds, then add the input state. */
void orc_chacha20_block(const uint32_t key[8], uint32_t counter,
                        const uint32_t nonce[3], uint32_t out[16]) {
    uint32_t s[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) s[4 + i] = key[i];
    s[12] = counter;
    s[13] = nonce[0]; s[14] = nonce[1]; s[15] = nonce[2];
    uint32_t x[16];
    memcpy(x, s, sizeof(x));
    for (int i = 0; i < 10; i++) {
        QR(x[0], x[4], x[8], x[12]);
        QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]);
        QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]);
        QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]);
        QR(x[3], x[4], x[9], x[14]);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/*
 * The project's random stream: ChaCha20 with
 *   key   = (seed mod 2^32, seed >> 32, domain, 0, 0, 0, 0, 0)
 *   nonce = (id0, id1, 0)
 * and block counter 0, 1, 2, ...; word k of the stream is word k%16 of block
 * k/16.  Writes words [0, n_words).
 */
void orc_stream_words(uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1,
                      uint32_t *out, size_t n_words) {
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), domain, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {id0, id1, 0};
    uint32_t blk[16];
    for (size_t b = 0; 16 * b < n_words; b++) {
        orc_chacha20_block(key, (uint32_t)b, nonce, blk);
        for (int i = 0; i < 16 && 16 * b + i < n_words; i++) out[16 * b + i] = blk[i];
    }
}

/* uniform residue mod q: coefficient k takes stream words 4k..4k+3 as one
 * 128-bit little-endian integer and reduces it mod q (bias < q / 2^128). */
void orc_sample_uniform(uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1,
                        uint64_t q, uint64_t *out, size_t n) {
    uint32_t *w = (uint32_t *)malloc(4 * n * sizeof(uint32_t));
    orc_stream_words(seed, domain, id0, id1, w, 4 * n);
    for (size_t k = 0; k < n; k++) {
        u128 v = (u128)w[4 * k] | ((u128)w[4 * k + 1] << 32) |
                 ((u128)w[4 * k + 2] << 64) | ((u128)w[4 * k + 3] << 96);
        out[k] = (uint64_t)(v % q);
    }
    free(w);
}

/* ternary {-1,0,1}: coefficient k takes word k, t = floor(w*3 / 2^32), s = t-1 */
void orc_sample_ternary(uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1,
                        int64_t *out, size_t n) {
    uint32_t *w = (uint32_t *)malloc(n * sizeof(uint32_t));
    orc_stream_words(seed, domain, id0, id1, w, n);
    for (size_t k = 0; k < n; k++) out[k] = (int64_t)(((uint64_t)w[k] * 3) >> 32) - 1;
    free(w);
}

/* centered binomial with eta = 21: coefficient k takes words 2k, 2k+1 and
 * returns popcount(low 21 bits of the first) - popcount(low 21 bits of the second) */
void orc_sample_cbd(uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1,
                    int64_t *out, size_t n) {
    uint32_t *w = (uint32_t *)malloc(2 * n * sizeof(uint32_t));
    orc_stream_words(seed, domain, id0, id1, w, 2 * n);
    for (size_t k = 0; k < n; k++) {
        int a = 0, b = 0;
        for (int i = 0; i < 21; i++) {
            a += (w[2 * k] >> i) & 1;
            b += (w[2 * k + 1] >> i) & 1;
        }
        out[k] = a - b;
    }
    free(w);
}

/* ----------------------------------------------------------- encoding */

/*
 * Slot encoding (Sec. 2.2: N/2 complex values -> a degree-N polynomial,
 * scaled by Delta and rounded).  With zeta = exp(i*pi/N), slot j sits at the
 * root zeta^(e_j), e_j = 5^j mod 2N, and the polynomial m has
 *     m(zeta^(e_j)) = z_j  (and the conjugate relation at zeta^(-e_j)).
 * Writing v_k = m_k + i*m_{k+N/2} (k < n = N/2), one has m(zeta^e_j) =
 * sum_k v_k zeta^(e_j*k), whose inverse is
 *     v_k = (1/n) zeta^(-k) sum_j z_j exp(-2*pi*i*k*t_j/n),  t_j = (e_j-1)/4.
 * This routine evaluates exactly that, in the fixed operation order below,
 * then rounds half away from zero:
 *   1. y[t_j] = z_j
 *   2. X = forward DFT of y (size n) by iterative radix-2 decimation in time:
 *      bit-reversal permutation, then for len = 2, 4, ..., n and each block,
 *      for k < len/2: ang = 2.0*M_PI*(double)k/(double)len,
 *      w = (cos(ang), -sin(ang)), v = a[k+len/2]*w, a[k] = u+v, a[k+len/2] = u-v
 *      (complex product (br*wr - bi*wi, br*wi + bi*wr)).
 *   3. ang = M_PI*(double)k/(double)N, (c, s) = (cos(ang), sin(ang));
 *      re = X_re*c + X_im*s, im = X_im*c - X_re*s  (that is X * zeta^-k);
 *      f = scale/(double)n; re = re*f, im = im*f.
 *   4. m_k = round(re), m_{k+n} = round(im), returned as doubles (integers
 *      of any size; those of magnitude 2^52 and above are already integral).
 */
void orc_encode(const double *z_re, const double *z_im, int logn, double scale, double *m) {
    size_t N = (size_t)1 << logn, n = N / 2;
    int logh = logn - 1;
    double *ar = (double *)malloc(n * sizeof(double));
    double *ai = (double *)malloc(n * sizeof(double));
    double *yr = (double *)malloc(n * sizeof(double));
    double *yi = (double *)malloc(n * sizeof(double));
    uint64_t e = 1, two_n = 2 * (uint64_t)N;
    for (size_t j = 0; j < n; j++) {
        size_t t = (size_t)((e - 1) / 4);
        yr[t] = z_re[j];
        yi[t] = z_im[j];
        e = (e * 5) % two_n;
    }
    for (size_t i = 0; i < n; i++) {
        size_t r = logh > 0 ? bitrev((uint32_t)i, logh) : 0;
        ar[r] = yr[i];
        ai[r] = yi[i];
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        size_t half = len / 2;
        for (size_t start = 0; start < n; start += len) {
            for (size_t k = 0; k < half; k++) {
                double ang = 2.0 * M_PI * (double)k / (double)len;
                double wr = cos(ang), wi = -sin(ang);
                double br = ar[start + k + half], bi = ai[start + k + half];
                double vr = br * wr - bi * wi;
                double vi = br * wi + bi * wr;
                double ur = ar[start + k], ui = ai[start + k];
                ar[start + k] = ur + vr;
                ai[start + k] = ui + vi;
                ar[start + k + half] = ur - vr;
                ai[start + k + half] = ui - vi;
            }
        }
    }
    double f = scale / (double)n;
    for (size_t k = 0; k < n; k++) {
        double ang = M_PI * (double)k / (double)N;
        double c = cos(ang), s = sin(ang);
        double re = ar[k] * c + ai[k] * s;
        double im = ai[k] * c - ar[k] * s;
        re = re * f;
        im = im * f;
        m[k] = round(re);
        m[k + n] = round(im);
    }
    free(ar); free(ai); free(yr); free(yi);
}

/* The same map by its O(N^2) definition (long double accumulation), unrounded:
 *   m_i = (2/N) * Re( sum_j z_j * zeta^(-e_j * i) ) * scale */
void orc_encode_naive(const double *z_re, const double *z_im, int logn, double scale,
                      double *m_real) {
    size_t N = (size_t)1 << logn, n = N / 2;
    uint64_t two_n = 2 * (uint64_t)N;
    for (size_t i = 0; i < N; i++) {
        long double acc = 0.0L;
        uint64_t e = 1;
        for (size_t j = 0; j < n; j++) {
            uint64_t ex = (e * (uint64_t)i) % two_n;       /* zeta^(-e*i) */
            long double ang = -(long double)M_PI * (long double)ex / (long double)N;
            acc += (long double)z_re[j] * cosl(ang) - (long double)z_im[j] * sinl(ang);
            e = (e * 5) % two_n;
        }
        m_real[i] = (double)(acc * 2.0L / (long double)N * (long double)scale);
    }
}
