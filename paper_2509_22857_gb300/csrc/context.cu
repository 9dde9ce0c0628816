// Context, tables, encoder and the client / primitive entry points of the C ABI.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "host.h"

static thread_local std::string g_err;

int fhe_fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

extern "C" const char *fhe_last_error(void) { return g_err.c_str(); }

extern "C" uint64_t fhe_kernel_launches(void) { return (uint64_t)fhe_launch_counter(); }

// ================================================================ host math

u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

bool h_is_prime(u64 n) {
    static const u64 witnesses[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : witnesses)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    for (u64 a : witnesses) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int i = 1; i < r && composite; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

std::vector<u64> h_gen_primes(int bits, int count, u64 two_n, const std::vector<u64> &taken) {
    std::vector<u64> out;
    const u64 top = 1ull << bits;
    for (u64 c = top - two_n + 1; (long long)out.size() < count && c > two_n; c -= two_n) {
        if (!h_is_prime(c)) continue;
        bool dup = false;
        for (u64 t : taken) dup |= (t == c);
        for (u64 t : out) dup |= (t == c);
        if (!dup) out.push_back(c);
    }
    return out;
}

u64 h_root_2n(u64 q, u64 two_n) {
    for (u64 g = 2;; g++)
        if (h_powmod(g, (q - 1) / 2, q) == q - 1) return h_powmod(g, (q - 1) / two_n, q);
}

u64 h_double_mod(double v, u64 q) {
    const double av = std::fabs(v);
    u64 r;
    if (av < 9223372036854775808.0) {
        r = (u64)(long long)av % q;
    } else {
        int e;
        const double mant = std::frexp(av, &e);
        const u64 mi = (u64)std::ldexp(mant, 53);
        r = h_mulmod(mi % q, h_powmod(2, (u64)(e - 53), q), q);
    }
    return (v < 0 && r) ? q - r : r;
}

static uint32_t h_brv(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// ================================================================ encoder
// The slot encoding m = round(scale * sigma^-1(z)) with slot j at zeta^(5^j),
// zeta = exp(i pi / N).  Writing v_k = m_k + i m_{k+n}, v = (1/n) zeta^-k
// DFT_n(y) with y[t_j] = z_j, t_j = (5^j mod 2N - 1)/4.  The floating-point
// operations are done in a fixed order (this file is compiled without FMA
// contraction): radix-2 decimation in time after a bit-reversal permutation;
// twiddle of a length-len stage at k is (cos a, -sin a), a = 2.0*M_PI*k/len;
// the twist multiplies by (c, -s), c + i s = exp(i M_PI k / N), then by
// scale/n; rounding is half away from zero.

void Encoder::init(int logn) {
    logN = logn;
    N = (size_t)1 << logn;
    n = N / 2;
    const int logh = logn - 1;
    fft_off.assign(logh + 2, 0);
    fft_re.clear();
    fft_im.clear();
    for (int s = 1; s <= logh; s++) {
        const size_t len = (size_t)1 << s;
        fft_off[s] = fft_re.size();
        for (size_t k = 0; k < len / 2; k++) {
            const double ang = 2.0 * M_PI * (double)k / (double)len;
            fft_re.push_back(std::cos(ang));
            fft_im.push_back(std::sin(ang));
        }
    }
    tw_c.resize(n);
    tw_s.resize(n);
    for (size_t k = 0; k < n; k++) {
        const double ang = M_PI * (double)k / (double)N;
        tw_c[k] = std::cos(ang);
        tw_s[k] = std::sin(ang);
    }
    slot_pos.resize(n);
    u64 e = 1;
    for (size_t j = 0; j < n; j++) {
        slot_pos[j] = (uint32_t)((e - 1) / 4);
        e = (e * 5) % (2 * (u64)N);
    }
    brv.resize(n);
    for (size_t i = 0; i < n; i++) brv[i] = logh > 0 ? h_brv((uint32_t)i, logh) : 0;
}

void Encoder::encode(const double *re, const double *im, size_t nz, double scale, double *m) const {
    std::vector<double> yr(n, 0.0), yi(n, 0.0), ar(n), ai(n);
    for (size_t j = 0; j < n; j++) {
        const double zr = j < nz ? re[j] : 0.0;
        const double zi = (j < nz && im) ? im[j] : 0.0;
        yr[slot_pos[j]] = zr;
        yi[slot_pos[j]] = zi;
    }
    for (size_t i = 0; i < n; i++) {
        ar[brv[i]] = yr[i];
        ai[brv[i]] = yi[i];
    }
    for (int s = 1; ((size_t)1 << s) <= n; s++) {
        const size_t len = (size_t)1 << s, half = len / 2;
        const double *cr = &fft_re[fft_off[s]], *ci = &fft_im[fft_off[s]];
        for (size_t st = 0; st < n; st += len) {
            for (size_t k = 0; k < half; k++) {
                const double wr = cr[k], wi = -ci[k];
                const double br = ar[st + k + half], bi = ai[st + k + half];
                const double vr = br * wr - bi * wi;
                const double vi = br * wi + bi * wr;
                const double ur = ar[st + k], ui = ai[st + k];
                ar[st + k] = ur + vr;
                ai[st + k] = ui + vi;
                ar[st + k + half] = ur - vr;
                ai[st + k + half] = ui - vi;
            }
        }
    }
    const double f = scale / (double)n;
    for (size_t k = 0; k < n; k++) {
        const double c = tw_c[k], s = tw_s[k];
        double r = ar[k] * c + ai[k] * s;
        double i = ai[k] * c - ar[k] * s;
        r = r * f;
        i = i * f;
        m[k] = std::round(r);
        m[k + n] = std::round(i);
    }
}

// z_j = sum_k (v_k zeta^k) exp(+2 pi i k t_j / n), v_k = (m_k + i m_{k+n}) / scale
void Encoder::decode(const double *m, double scale, double *re, double *im, size_t nz) const {
    std::vector<double> xr(n), xi(n), ar(n), ai(n);
    for (size_t k = 0; k < n; k++) {
        const double vr = m[k] / scale, vi = m[k + n] / scale;
        xr[k] = vr * tw_c[k] - vi * tw_s[k];
        xi[k] = vr * tw_s[k] + vi * tw_c[k];
    }
    for (size_t i = 0; i < n; i++) {
        ar[brv[i]] = xr[i];
        ai[brv[i]] = xi[i];
    }
    for (int s = 1; ((size_t)1 << s) <= n; s++) {
        const size_t len = (size_t)1 << s, half = len / 2;
        const double *cr = &fft_re[fft_off[s]], *ci = &fft_im[fft_off[s]];
        for (size_t st = 0; st < n; st += len) {
            for (size_t k = 0; k < half; k++) {
                const double wr = cr[k], wi = ci[k];
                const double br = ar[st + k + half], bi = ai[st + k + half];
                const double vr = br * wr - bi * wi, vi = br * wi + bi * wr;
                const double ur = ar[st + k], ui = ai[st + k];
                ar[st + k] = ur + vr;
                ai[st + k] = ui + vi;
                ar[st + k + half] = ur - vr;
                ai[st + k + half] = ui - vi;
            }
        }
    }
    for (size_t j = 0; j < nz && j < n; j++) {
        re[j] = ar[slot_pos[j]];
        if (im) im[j] = ai[slot_pos[j]];
    }
}

// ================================================================ memory

cudaError_t pool_trim() {
    int dev = 0;
    cudaMemPool_t pool;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    return e;
}

int dev_alloc(fhe_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (ctx && ctx->fail_alloc_after.load() >= 0 && ctx->fail_alloc_after.fetch_sub(1) == 0)
        return fhe_fail(FHE_E_OOM, "device allocation refused (injected failure)");
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        // the stream-ordered pool may hold freed memory: return it and retry
        cudaGetLastError();
        if (pool_trim() == cudaSuccess) e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fhe_fail(FHE_E_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return FHE_OK;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

int ws_reserve(fhe_ctx *ctx, u64 **ws, size_t *have, size_t words) {
    if (*have >= words) return FHE_OK;
    FHE_CU(cudaDeviceSynchronize());
    dev_free(*ws);
    *ws = nullptr;
    *have = 0;
    void *p;
    FHE_TRY(dev_alloc(ctx, &p, words * 8));
    *ws = (u64 *)p;
    *have = words;
    return FHE_OK;
}

static int upload(fhe_ctx *ctx, const void *host, size_t bytes, void **dev) {
    FHE_TRY(dev_alloc(ctx, dev, bytes));
    ctx->owned.push_back(*dev);
    FHE_CU(cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice));
    return FHE_OK;
}

int galois_of_step(const fhe_ctx *ctx, int step) {
    const long long n = ctx->N / 2;
    long long r = ((step % n) + n) % n;
    return (int)h_powmod(5, (u64)r, 2 * (u64)ctx->N);
}

size_t key_words(const fhe_ctx *ctx) {
    const int digits = (ctx->L + ctx->alpha) / ctx->alpha;
    return (size_t)digits * 2 * ctx->n_primes * ctx->N;
}

// ================================================================ context

static int build_tables(fhe_ctx *c) {
    const int np = c->n_primes, L = c->L, al = c->alpha;
    const u64 N = (u64)c->N;
    std::vector<PrimeTab> pt(np);
    for (int t = 0; t < np; t++) {
        const u64 q = c->primes[t];
        int b = 64 - __builtin_clzll(q);
        pt[t].m.q = q;
        pt[t].m.b = b;
        pt[t].m.mu = (u64)(((u128)1 << (b + 62)) / q);
        const u64 psi = h_root_2n(q, 2 * N), psi_inv = h_invmod(psi, q);
        std::vector<u64> pw(N), pwi(N);
        pw[0] = pwi[0] = 1;
        for (u64 e = 1; e < N; e++) {
            pw[e] = h_mulmod(pw[e - 1], psi, q);
            pwi[e] = h_mulmod(pwi[e - 1], psi_inv, q);
        }
        std::vector<ulonglong2> fw(N), iv(N);
        for (u64 k = 0; k < N; k++) {
            const u64 w = pw[h_brv((uint32_t)k, c->logN)], wi = pwi[h_brv((uint32_t)k, c->logN)];
            fw[k] = make_ulonglong2(w, h_shoup(w, q));
            iv[k] = make_ulonglong2(wi, h_shoup(wi, q));
        }
        void *d;
        FHE_TRY(upload(c, fw.data(), N * sizeof(ulonglong2), &d));
        pt[t].fwd = (const ulonglong2 *)d;
        FHE_TRY(upload(c, iv.data(), N * sizeof(ulonglong2), &d));
        pt[t].inv = (const ulonglong2 *)d;
        pt[t].n_inv = h_invmod(N % q, q);
        pt[t].n_inv_sh = h_shoup(pt[t].n_inv, q);
    }
    void *d;
    FHE_TRY(upload(c, pt.data(), np * sizeof(PrimeTab), &d));
    c->dc.primes = (const PrimeTab *)d;
    c->dc.logN = c->logN;
    c->dc.L = L;
    c->dc.alpha = al;
    c->dc.logR1 = (c->logN + 1) / 2;
    c->dc.logR2 = c->logN / 2;

    // ModDown constants: P = prod p_m
    std::vector<ulonglong2> zs(al);
    std::vector<u64> za(al), phat((size_t)al * (L + 1)), halfp(L + 1);
    std::vector<ulonglong2> pinv(L + 1);
    for (int m = 0; m < al; m++) {
        const u64 p = c->primes[L + 1 + m];
        u64 ph = 1;
        for (int u = 0; u < al; u++)
            if (u != m) ph = h_mulmod(ph, c->primes[L + 1 + u] % p, p);
        const u64 phi = h_invmod(ph, p);
        const u64 sc = h_mulmod(h_invmod(N % p, p), phi, p);
        zs[m] = make_ulonglong2(sc, h_shoup(sc, p));
        za[m] = h_mulmod((p - 1) / 2, phi, p);   // floor(P/2) = (P-1)/2 = (p-1)/2 mod p
        for (int i = 0; i <= L; i++) {
            const u64 q = c->primes[i];
            u64 v = 1;
            for (int u = 0; u < al; u++)
                if (u != m) v = h_mulmod(v, c->primes[L + 1 + u] % q, q);
            phat[(size_t)m * (L + 1) + i] = v;
        }
    }
    for (int i = 0; i <= L; i++) {
        const u64 q = c->primes[i];
        u64 pm = 1;
        for (int u = 0; u < al; u++) pm = h_mulmod(pm, c->primes[L + 1 + u] % q, q);
        // floor(P/2) = (P-1)/2 mod q
        halfp[i] = h_mulmod((pm + q - 1) % q, h_invmod(2, q), q);
        const u64 inv = h_invmod(pm, q);
        pinv[i] = make_ulonglong2(inv, h_shoup(inv, q));
    }
    FHE_TRY(upload(c, zs.data(), al * sizeof(ulonglong2), &d));
    c->dc.md_z_scale = (const ulonglong2 *)d;
    FHE_TRY(upload(c, za.data(), al * 8, &d));
    c->dc.md_z_add = (const u64 *)d;
    FHE_TRY(upload(c, phat.data(), phat.size() * 8, &d));
    c->dc.md_phat = (const u64 *)d;
    FHE_TRY(upload(c, halfp.data(), halfp.size() * 8, &d));
    c->dc.md_halfp = (const u64 *)d;
    FHE_TRY(upload(c, pinv.data(), pinv.size() * sizeof(ulonglong2), &d));
    c->dc.md_pinv = (const ulonglong2 *)d;
    // exact ModDown: fixed-point weights 2^E / p_m and P mod q_i
    int min_bits = 64;
    for (int m = 0; m < al; m++) min_bits = std::min(min_bits, 64 - __builtin_clzll(c->primes[L + 1 + m]));
    const int E = 63 + min_bits;
    std::vector<u64> mw(al), pmod(L + 1);
    for (int m = 0; m < al; m++) mw[m] = (u64)(((unsigned __int128)1 << E) / c->primes[L + 1 + m]);
    for (int i = 0; i <= L; i++) {
        const u64 q = c->primes[i];
        u64 pm = 1;
        for (int u = 0; u < al; u++) pm = h_mulmod(pm, c->primes[L + 1 + u] % q, q);
        pmod[i] = pm;
    }
    c->dc.md_E = E;
    FHE_TRY(upload(c, mw.data(), al * 8, &d));
    c->dc.md_w = (const u64 *)d;
    FHE_TRY(upload(c, pmod.data(), pmod.size() * 8, &d));
    c->dc.md_pmod = (const u64 *)d;

    // per-level tables
    c->lt.resize(L + 1);
    for (int lv = 0; lv <= L; lv++) {
        LevelTab &T = c->lt[lv];
        T.level = lv;
        T.n_digits = (lv + al) / al;
        T.ext = lv + 1 + al;
        std::vector<ulonglong2> ys(lv + 1);
        std::vector<u64> hat((size_t)T.n_digits * al * T.ext, 0);
        for (int j = 0; j < T.n_digits; j++) {
            const int lo = j * al, hi = std::min(lo + al, lv + 1);
            for (int i = lo; i < hi; i++) {
                const u64 q = c->primes[i];
                u64 h = 1;
                for (int u = lo; u < hi; u++)
                    if (u != i) h = h_mulmod(h, c->primes[u] % q, q);
                const u64 v = h_mulmod(h_invmod(N % q, q), h_invmod(h, q), q);
                ys[i] = make_ulonglong2(v, h_shoup(v, q));
                for (int t = 0; t < T.ext; t++) {
                    const u64 pt_ = c->primes[ext_prime(t, lv, L)];
                    u64 hh = 1;
                    for (int u = lo; u < hi; u++)
                        if (u != i) hh = h_mulmod(hh, c->primes[u] % pt_, pt_);
                    hat[((size_t)j * al + (i - lo)) * T.ext + t] = hh;
                }
            }
        }
        FHE_TRY(upload(c, ys.data(), ys.size() * sizeof(ulonglong2), &d));
        T.y_scale = (const ulonglong2 *)d;
        FHE_TRY(upload(c, hat.data(), hat.size() * 8, &d));
        T.modup_hat = (const u64 *)d;
        std::vector<ulonglong2> qi(std::max(lv, 1));
        std::vector<u64> qm(std::max(lv, 1));
        for (int i = 0; i < lv; i++) {
            const u64 q = c->primes[i], ql = c->primes[lv];
            const u64 inv = h_invmod(ql % q, q);
            qi[i] = make_ulonglong2(inv, h_shoup(inv, q));
            qm[i] = ql % q;
        }
        FHE_TRY(upload(c, qi.data(), qi.size() * sizeof(ulonglong2), &d));
        T.q_last_inv = (const ulonglong2 *)d;
        FHE_TRY(upload(c, qm.data(), qm.size() * 8, &d));
        T.q_last_mod = (const u64 *)d;
    }
    return FHE_OK;
}

extern "C" int fhe_ctx_create(const fhe_params *p, fhe_ctx **out) {
    if (!p || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (p->log_n < 12 || p->log_n > 16) return fhe_fail(FHE_E_INVAL, "log_n must be in [12, 16]");
    if (p->alpha < 1 || p->alpha > 8) return fhe_fail(FHE_E_INVAL, "alpha must be in [1, 8]");
    if (p->L < 0 || p->L + 1 + p->alpha > FHE_MAX_LIMBS) return fhe_fail(FHE_E_INVAL, "too many primes");
    const u64 two_n = 2ull << p->log_n;
    const int n_primes = p->L + 1 + p->alpha;
    int max_bits = 0;
    if (p->primes) {
        // 58: lazy NTT values stay below 2^61 and Barrett's constants fit 64 bits
        for (int i = 0; i < n_primes; i++) {
            const u64 q = p->primes[i];
            const int b = q ? 64 - __builtin_clzll(q) : 0;
            if (b < 20 || b > 58) return fhe_fail(FHE_E_INVAL, "explicit primes must have 20..58 bits");
            if (q % two_n != 1) return fhe_fail(FHE_E_INVAL, "explicit prime not = 1 mod 2N: " + std::to_string(q));
            if (!h_is_prime(q)) return fhe_fail(FHE_E_INVAL, "explicit chain value is not prime: " + std::to_string(q));
            for (int j = 0; j < i; j++)
                if (p->primes[j] == q) return fhe_fail(FHE_E_INVAL, "explicit chain repeats a prime");
            max_bits = std::max(max_bits, b);
        }
    } else {
        // 31..58 bits for generated chains
        if (p->q_bits > 58 || p->q0_bits > 58 || p->p_bits > 58 || p->q_bits < 31 || p->q0_bits < 31 ||
            p->p_bits < 31)
            return fhe_fail(FHE_E_INVAL, "prime sizes must be in [31, 58] bits");
        max_bits = std::max(std::max(p->q_bits, p->q0_bits), p->p_bits);
    }
    // the key inner product sums one product below 2^(2b) per digit; Barrett
    // reduction takes sums below 2^(b+62)
    const int digits_top = (p->L + p->alpha) / p->alpha;
    if ((long long)digits_top > (1ll << (62 - max_bits)))
        return fhe_fail(FHE_E_INVAL, std::to_string(digits_top) + " key-switching digits exceed 2^(62 - " +
                                         std::to_string(max_bits) + ")");
    int ndev = 0;
    FHE_CU(cudaGetDeviceCount(&ndev));
    if (p->device < 0 || p->device >= ndev) return fhe_fail(FHE_E_INVAL, "no such CUDA device");
    FHE_CU(cudaSetDevice(p->device));
    {
        // Temporaries of a step come from the device's stream-ordered pool.
        // Keep what the pool has mapped across synchronisations (its default
        // gives everything back at each one, and the next batch maps it
        // again); dev_alloc trims the pool when a plain allocation is refused.
        // The setting belongs to this process's context only.
        cudaMemPool_t pool;
        FHE_CU(cudaDeviceGetDefaultMemPool(&pool, p->device));
        uint64_t keep = UINT64_MAX;
        FHE_CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    std::unique_ptr<fhe_ctx> c(new fhe_ctx());
    c->prm = *p;
    c->dev = p->device;
    c->logN = p->log_n;
    c->N = 1ll << p->log_n;
    c->L = p->L;
    c->alpha = p->alpha;
    c->n_primes = p->L + 1 + p->alpha;
    c->scale = std::pow(2.0, p->log_scale);
    c->prm.primes = nullptr;   // the caller's array is read during this call only
    if (p->primes) {
        c->primes.assign(p->primes, p->primes + n_primes);
    } else {
        std::vector<u64> rest = p->L > 0 ? h_gen_primes(p->q_bits, p->L, two_n, {}) : std::vector<u64>();
        if ((int)rest.size() != p->L) return fhe_fail(FHE_E_INVAL, "not enough q primes");
        std::vector<u64> q0 = h_gen_primes(p->q0_bits, 1, two_n, rest);
        if (q0.size() != 1) return fhe_fail(FHE_E_INVAL, "no q0 prime");
        std::vector<u64> taken = rest;
        taken.push_back(q0[0]);
        std::vector<u64> sp = h_gen_primes(p->p_bits, p->alpha, two_n, taken);
        if ((int)sp.size() != p->alpha) return fhe_fail(FHE_E_INVAL, "not enough special primes");
        c->primes.push_back(q0[0]);
        for (u64 x : rest) c->primes.push_back(x);
        for (u64 x : sp) c->primes.push_back(x);
    }
    c->enc.init(c->logN);
    int r = build_tables(c.get());
    // the tables' uploads complete before any stream of the caller uses them
    if (r == FHE_OK && cudaDeviceSynchronize() != cudaSuccess)
        r = fhe_fail(FHE_E_CUDA, std::string("table upload: ") + cudaGetErrorString(cudaGetLastError()));
    if (r != FHE_OK) {
        for (void *q : c->owned) dev_free(q);
        return r;
    }
    *out = c.release();
    return FHE_OK;
}

extern "C" int fhe_ctx_destroy(fhe_ctx *ctx) {
    if (!ctx) return FHE_OK;
    cudaSetDevice(ctx->dev);
    cudaDeviceSynchronize();
    for (void *p : ctx->owned) dev_free(p);
    dev_free(ctx->ks_ws);
    dev_free(ctx->rs_ws);
    delete ctx;
    return FHE_OK;
}

extern "C" int fhe_ctx_inject_alloc_failure(fhe_ctx *ctx, int after) {
    if (!ctx) return fhe_fail(FHE_E_INVAL, "null argument");
    ctx->fail_alloc_after.store(after < 0 ? -1 : after);
    return FHE_OK;
}

extern "C" int fhe_ctx_set_linear_chunk(fhe_ctx *ctx, int lin_chunk_srcs) {
    if (!ctx || lin_chunk_srcs < 2) return fhe_fail(FHE_E_INVAL, "linear chunk must be at least 2 sources");
    ctx->lin_chunk_srcs = lin_chunk_srcs;
    return FHE_OK;
}

extern "C" int fhe_ctx_set_encode_scratch(fhe_ctx *ctx, size_t bytes) {
    if (!ctx || bytes == 0) return fhe_fail(FHE_E_INVAL, "bad argument");
    ctx->on_demand_bytes = bytes;
    return FHE_OK;
}

extern "C" int fhe_ctx_set_keyswitch_batch(fhe_ctx *ctx, int max_items) {
    if (!ctx || max_items < 0) return fhe_fail(FHE_E_INVAL, "bad argument");
    ctx->ks_item_cap = max_items;
    return FHE_OK;
}

extern "C" int fhe_ctx_set_mac_images(fhe_ctx *ctx, int images_per_cta) {
    if (!ctx || !(images_per_cta == 0 || images_per_cta == 1 || images_per_cta == 2 || images_per_cta == 4 ||
                  images_per_cta == 8))
        return fhe_fail(FHE_E_INVAL, "images per MAC block must be 0, 1, 2, 4 or 8");
    ctx->mac_images = images_per_cta;
    return FHE_OK;
}

extern "C" int fhe_ctx_primes(const fhe_ctx *ctx, uint64_t *out, size_t cap, size_t *n) {
    if (!ctx || !n) return fhe_fail(FHE_E_INVAL, "null argument");
    *n = ctx->primes.size();
    if (out) {
        if (cap < ctx->primes.size()) return fhe_fail(FHE_E_INVAL, "buffer too small");
        for (size_t i = 0; i < ctx->primes.size(); i++) out[i] = ctx->primes[i];
    }
    return FHE_OK;
}

// ================================================================ core ops

int op_ntt(fhe_ctx *ctx, const u64 *src, u64 *dst, long long item, int n_items, int n_limbs,
           const unsigned char *pidx, bool inverse, cudaStream_t s) {
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.dst = dst;
    a.src_item = a.dst_item = item;
    a.n_items = n_items;
    a.n_limbs = n_limbs;
    for (int l = 0; l < n_limbs; l++) a.pidx[l] = pidx ? pidx[l] : (unsigned char)l;
    FHE_CU(launch_ntt(ctx->dc, a, inverse, s));
    return FHE_OK;
}

int op_ks_ip_babies(fhe_ctx *ctx, KsArgs a, const IpBabies &bb, cudaStream_t s, u64 *ws) {
    const size_t per = ks_workspace_words(ctx->dc, a.level);
    if (!ws) {
        // the ModUp that filled it reserved the same size: no reallocation here
        if (ctx->ks_ws_words < per * (size_t)a.n_items)
            return fhe_fail(FHE_E_INVAL, "internal: baby-step inner products without their ModUp");
        ws = ctx->ks_ws;
    }
    a.ws = ws;
    a.ws_item = (long long)per;
    FHE_CU(launch_ks_ip_babies(ctx->dc, ctx->lt[a.level], a, bb, s));
    return FHE_OK;
}

int op_keyswitch(fhe_ctx *ctx, KsArgs a, cudaStream_t s, u64 *ws, int phases) {
    const size_t per = ks_workspace_words(ctx->dc, a.level);
    if (!ws) {
        FHE_TRY(ws_reserve(ctx, &ctx->ks_ws, &ctx->ks_ws_words, per * (size_t)a.n_items));
        ws = ctx->ks_ws;
    }
    a.ws = ws;
    a.ws_item = (long long)per;
    FHE_CU(launch_keyswitch(ctx->dc, ctx->lt[a.level], a, s, nullptr, phases));
    return FHE_OK;
}

int op_rescale(fhe_ctx *ctx, const u64 *in, long long in_item, u64 *out, long long out_item, int n_items,
               int n_poly, int level, cudaStream_t s, u64 *ws) {
    if (level < 1) return fhe_fail(FHE_E_LEVEL, "rescale at level 0");
    if (!ws) {
        FHE_TRY(ws_reserve(ctx, &ctx->rs_ws, &ctx->rs_ws_words, (size_t)n_items * n_poly * ctx->N));
        ws = ctx->rs_ws;
    }
    RescaleArgs a;
    a.in = in;
    a.in_item = in_item;
    a.out = out;
    a.out_item = out_item;
    a.n_items = n_items;
    a.n_poly = n_poly;
    a.level = level;
    a.ws = ws;
    FHE_CU(launch_rescale(ctx->dc, ctx->lt[level], a, s));
    return FHE_OK;
}

int enc_tables(fhe_ctx *ctx, const EncTab **out) {
    if (!ctx->enc_dev_ready) {
        const Encoder &E = ctx->enc;
        EncTab t;
        memset(&t, 0, sizeof(t));
        void *d;
        FHE_TRY(upload(ctx, E.fft_re.data(), E.fft_re.size() * sizeof(double), &d));
        t.fft_re = (const double *)d;
        FHE_TRY(upload(ctx, E.fft_im.data(), E.fft_im.size() * sizeof(double), &d));
        t.fft_im = (const double *)d;
        for (size_t st = 0; st < E.fft_off.size() && st < 24; st++) t.off[st] = (long long)E.fft_off[st];
        FHE_TRY(upload(ctx, E.tw_c.data(), E.tw_c.size() * sizeof(double), &d));
        t.tw_c = (const double *)d;
        FHE_TRY(upload(ctx, E.tw_s.data(), E.tw_s.size() * sizeof(double), &d));
        t.tw_s = (const double *)d;
        std::vector<unsigned> perm(E.n);
        for (size_t j = 0; j < E.n; j++) perm[j] = E.brv[E.slot_pos[j]];
        FHE_TRY(upload(ctx, perm.data(), perm.size() * sizeof(unsigned), &d));
        t.perm = (const unsigned *)d;
        FHE_CU(cudaDeviceSynchronize());
        ctx->enc_dev = t;
        ctx->enc_dev_ready = true;
    }
    *out = &ctx->enc_dev;
    return FHE_OK;
}

int op_encode_to(fhe_ctx *ctx, const double *m_host, int level, u64 *dst, cudaStream_t s, bool ext) {
    const int n_limbs = level + 1 + (ext ? ctx->alpha : 0);
    std::vector<unsigned char> pidx(n_limbs);
    for (int l = 0; l < n_limbs; l++) pidx[l] = (unsigned char)ext_prime(l, ext ? level : ctx->L, ctx->L);
    double *dm;
    FHE_ALLOC_ASYNC(&dm, ctx->N * sizeof(double), s);
    FHE_CU(cudaMemcpyAsync(dm, m_host, ctx->N * sizeof(double), cudaMemcpyHostToDevice, s));
    FHE_CU(launch_double_to_limbs(ctx->dc, dm, dst, n_limbs, s, ext ? level : -1));
    FHE_CU(cudaFreeAsync(dm, s));
    FHE_TRY(op_ntt(ctx, dst, dst, 0, 1, n_limbs, pidx.data(), false, s));
    return FHE_OK;
}

// ================================================================ keys

enum { DOM_SECRET = 1, DOM_KEY_A = 2, DOM_KEY_E = 3, DOM_ENC_A = 4, DOM_ENC_E = 5 };

static int make_switch_key(fhe_ctx *c, uint64_t seed, int key_id, const u64 *s_ntt, const u64 *s_new, u64 *key) {
    const int np = c->n_primes, al = c->alpha, L = c->L;
    const long long N = c->N;
    const int digits = (L + al) / al;
    std::vector<unsigned char> pidx(np);
    for (int t = 0; t < np; t++) pidx[t] = (unsigned char)t;
    // P mod q_t for every Q prime
    std::vector<u64> pmod(np, 0);
    for (int t = 0; t <= L; t++) {
        u64 v = 1;
        for (int u = 0; u < al; u++) v = h_mulmod(v, c->primes[L + 1 + u] % c->primes[t], c->primes[t]);
        pmod[t] = v;
    }
    u64 *d_pmod;
    FHE_TRY(dev_alloc(c, (void **)&d_pmod, np * 8));
    long long *e;
    FHE_TRY(dev_alloc(c, (void **)&e, N * 8));
    FHE_CU(cudaMemcpy(d_pmod, pmod.data(), np * 8, cudaMemcpyHostToDevice));
    for (int j = 0; j < digits; j++) {
        u64 *b = key + (size_t)(2 * j) * np * N;
        u64 *a = key + (size_t)(2 * j + 1) * np * N;
        FHE_CU(launch_sample_uniform(c->dc, seed, DOM_KEY_A, (uint32_t)key_id, (uint32_t)j * 65536u, 1, a, np,
                                     pidx.data(), 0));
        FHE_CU(launch_sample_small(c->dc, seed, DOM_KEY_E, (uint32_t)key_id, (uint32_t)j, 1, e, 0));
        FHE_CU(launch_signed_to_limbs(c->dc, e, b, np, pidx.data(), 0));
        FHE_TRY(op_ntt(c, b, b, 0, 1, np, pidx.data(), false, 0));
        // b = e - a*s
        FHE_CU(launch_mul_limbs(c->dc, a, s_ntt, b, 1, b, np, pidx.data(), 0));
        // + (P mod q_t) * s_new[t] on the digit's own limbs
        const int lo = j * al, hi = std::min(lo + al, L + 1);
        FHE_CU(launch_axpy_limbs(c->dc, s_new + (size_t)lo * N, d_pmod + lo, b + (size_t)lo * N, hi - lo,
                                 pidx.data() + lo, 0));
    }
    FHE_CU(cudaDeviceSynchronize());
    dev_free(d_pmod);
    dev_free(e);
    return FHE_OK;
}

extern "C" int fhe_keygen(fhe_ctx *c, uint64_t seed, const int32_t *rot_steps, size_t n_steps, fhe_sk **sk_out,
                          fhe_evk **evk_out) {
    if (!c || !sk_out || !evk_out || (n_steps && !rot_steps)) return fhe_fail(FHE_E_INVAL, "null argument");
    FHE_CU(cudaSetDevice(c->dev));
    const int np = c->n_primes;
    const long long N = c->N;
    std::vector<unsigned char> pidx(np);
    for (int t = 0; t < np; t++) pidx[t] = (unsigned char)t;
    std::unique_ptr<fhe_sk> sk(new fhe_sk());
    sk->ctx = c;
    FHE_TRY(dev_alloc(c, (void **)&sk->s_ntt, (size_t)np * N * 8));
    long long *scoef;
    FHE_TRY(dev_alloc(c, (void **)&scoef, N * 8));
    FHE_CU(launch_sample_small(c->dc, seed, DOM_SECRET, 0, 0, 0, scoef, 0));
    FHE_CU(launch_signed_to_limbs(c->dc, scoef, sk->s_ntt, np, pidx.data(), 0));
    FHE_TRY(op_ntt(c, sk->s_ntt, sk->s_ntt, 0, 1, np, pidx.data(), false, 0));
    FHE_CU(cudaDeviceSynchronize());
    dev_free(scoef);

    std::unique_ptr<fhe_evk> evk(new fhe_evk());
    evk->ctx = c;
    evk->digits = (c->L + c->alpha) / c->alpha;
    const size_t kw = key_words(c);
    u64 *s2;
    FHE_TRY(dev_alloc(c, (void **)&s2, (size_t)np * N * 8));
    FHE_CU(launch_mul_limbs(c->dc, sk->s_ntt, sk->s_ntt, nullptr, 0, s2, np, pidx.data(), 0));
    FHE_TRY(dev_alloc(c, (void **)&evk->relin, kw * 8));
    FHE_TRY(make_switch_key(c, seed, 0, sk->s_ntt, s2, evk->relin));
    for (size_t i = 0; i < n_steps; i++) {
        const int k = galois_of_step(c, rot_steps[i]);
        if (k == 1 || evk->galois.count(k)) continue;
        FHE_CU(launch_automorphism(c->dc, sk->s_ntt, s2, np, k, 0));
        u64 *key;
        FHE_TRY(dev_alloc(c, (void **)&key, kw * 8));
        evk->galois[k] = key;
        FHE_TRY(make_switch_key(c, seed, k, sk->s_ntt, s2, key));
    }
    FHE_CU(cudaDeviceSynchronize());
    dev_free(s2);
    *sk_out = sk.release();
    *evk_out = evk.release();
    return FHE_OK;
}

extern "C" int fhe_sk_free(fhe_sk *sk) {
    if (!sk) return FHE_OK;
    cudaDeviceSynchronize();
    dev_free(sk->s_ntt);
    delete sk;
    return FHE_OK;
}

extern "C" int fhe_evk_free(fhe_evk *evk) {
    if (!evk) return FHE_OK;
    cudaDeviceSynchronize();
    dev_free(evk->relin);
    for (auto &kv : evk->galois) dev_free(kv.second);
    delete evk;
    return FHE_OK;
}

// every residue of n_blocks blocks laid out [block][L+1+alpha][N] below its prime
static bool limbs_in_range(const fhe_ctx *c, const uint64_t *buf, size_t n_blocks) {
    for (size_t b = 0; b < n_blocks; b++)
        for (int t = 0; t < c->n_primes; t++) {
            const u64 q = c->primes[t];
            const uint64_t *p = buf + (b * c->n_primes + t) * (size_t)c->N;
            for (long long i = 0; i < c->N; i++)
                if (p[i] >= q) return false;
        }
    return true;
}

extern "C" int fhe_sk_import(fhe_ctx *c, const uint64_t *buf, size_t n_words, fhe_sk **out) {
    if (!c || !buf || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    const size_t w = (size_t)c->n_primes * c->N;
    if (n_words != w) return fhe_fail(FHE_E_INVAL, "a secret key has (L+1+alpha)*N words");
    if (!limbs_in_range(c, buf, 1)) return fhe_fail(FHE_E_INVAL, "secret key residue not below its prime");
    FHE_CU(cudaSetDevice(c->dev));
    std::unique_ptr<fhe_sk> sk(new fhe_sk());
    sk->ctx = c;
    FHE_TRY(dev_alloc(c, (void **)&sk->s_ntt, w * 8));
    // synchronised: a pageable upload may return before its DMA lands, and
    // the key is then used from other (non-blocking) streams
    cudaError_t e = cudaMemcpy(sk->s_ntt, buf, w * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dev_free(sk->s_ntt);
        return fhe_fail(FHE_E_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    }
    *out = sk.release();
    return FHE_OK;
}

extern "C" int fhe_evk_import(fhe_ctx *c, const int32_t *galois, size_t n_keys, const uint64_t *const *keys,
                              size_t words_per_key, fhe_evk **out) {
    if (!c || !out || (n_keys && (!galois || !keys))) return fhe_fail(FHE_E_INVAL, "null argument");
    const size_t kw = key_words(c);
    if (words_per_key != kw) return fhe_fail(FHE_E_INVAL, "key size does not match the context");
    const int digits = (c->L + c->alpha) / c->alpha;
    int n_relin = 0;
    std::map<int, size_t> seen;
    for (size_t i = 0; i < n_keys; i++) {
        const int k = galois[i];
        if (!keys[i]) return fhe_fail(FHE_E_INVAL, "null key buffer");
        if (k == 0) {
            n_relin++;
            continue;
        }
        if (k < 3 || (long long)k >= 2 * c->N || (k & 1) == 0)
            return fhe_fail(FHE_E_INVAL, "not a Galois element of this ring: " + std::to_string(k));
        if (!seen.emplace(k, i).second) return fhe_fail(FHE_E_INVAL, "duplicate Galois element " + std::to_string(k));
    }
    if (n_relin != 1) return fhe_fail(FHE_E_INVAL, "exactly one relinearisation key (galois 0) is required");
    for (size_t i = 0; i < n_keys; i++)
        if (!limbs_in_range(c, keys[i], (size_t)digits * 2))
            return fhe_fail(FHE_E_INVAL, "key " + std::to_string(i) + ": residue not below its prime");
    FHE_CU(cudaSetDevice(c->dev));
    fhe_evk *evk = new fhe_evk();
    evk->ctx = c;
    evk->digits = digits;
    int rc = FHE_OK;
    for (size_t i = 0; i < n_keys && rc == FHE_OK; i++) {
        u64 *d = nullptr;
        rc = dev_alloc(c, (void **)&d, kw * 8);
        if (rc != FHE_OK) break;
        if (galois[i] == 0)
            evk->relin = d;
        else
            evk->galois[galois[i]] = d;
        const cudaError_t e = cudaMemcpy(d, keys[i], kw * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = fhe_fail(FHE_E_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    }
    // as for the secret key: the uploads complete before the keys are used
    if (rc == FHE_OK) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fhe_fail(FHE_E_CUDA, std::string("key upload: ") + cudaGetErrorString(e));
    }
    if (rc != FHE_OK) {
        fhe_evk_free(evk);
        return rc;
    }
    *out = evk;
    return FHE_OK;
}

extern "C" int fhe_evk_galois(const fhe_evk *evk, int32_t *out, size_t cap, size_t *n) {
    if (!evk || !n) return fhe_fail(FHE_E_INVAL, "null argument");
    *n = evk->galois.size();
    if (out) {
        if (cap < evk->galois.size()) return fhe_fail(FHE_E_INVAL, "buffer too small");
        size_t i = 0;
        for (auto &kv : evk->galois) out[i++] = kv.first;
    }
    return FHE_OK;
}

// ================================================================ encode / encrypt

extern "C" int fhe_encode(fhe_ctx *c, const double *re, const double *im, size_t n, double scale, int level,
                          fhe_pt **out) {
    if (!c || !out || (n && !re)) return fhe_fail(FHE_E_INVAL, "null argument");
    if (n > (size_t)c->N / 2) return fhe_fail(FHE_E_INVAL, "more slots than N/2");
    if (level < 0 || level > c->L) return fhe_fail(FHE_E_LEVEL, "level out of range");
    if (!(scale > 0)) return fhe_fail(FHE_E_INVAL, "scale must be positive");
    FHE_CU(cudaSetDevice(c->dev));
    std::vector<double> m(c->N);
    c->enc.encode(re, im, n, scale, m.data());
    std::unique_ptr<fhe_pt> pt(new fhe_pt());
    pt->ctx = c;
    pt->level = level;
    pt->scale = scale;
    FHE_TRY(dev_alloc(c, (void **)&pt->d, (size_t)(level + 1) * c->N * 8));
    FHE_TRY(op_encode_to(c, m.data(), level, pt->d, 0));
    FHE_CU(cudaDeviceSynchronize());
    *out = pt.release();
    return FHE_OK;
}

extern "C" int fhe_encode_coeffs(fhe_ctx *c, const double *re, const double *im, size_t n, double scale,
                                 double *out) {
    if (!c || !out || (n && !re)) return fhe_fail(FHE_E_INVAL, "null argument");
    if (n > (size_t)c->N / 2) return fhe_fail(FHE_E_INVAL, "more slots than N/2");
    c->enc.encode(re, im, n, scale, out);
    return FHE_OK;
}

extern "C" int fhe_pt_free(fhe_pt *pt) {
    if (!pt) return FHE_OK;
    cudaDeviceSynchronize();
    dev_free(pt->d);
    delete pt;
    return FHE_OK;
}

extern "C" int fhe_encrypt(fhe_ctx *c, const fhe_sk *sk, const fhe_pt *pt, uint64_t seed, fhe_ct **out) {
    if (!c || !sk || !pt || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    FHE_CU(cudaSetDevice(c->dev));
    const int lv = pt->level, nl = lv + 1;
    const long long N = c->N;
    std::vector<unsigned char> pidx(nl);
    for (int t = 0; t < nl; t++) pidx[t] = (unsigned char)t;
    std::unique_ptr<fhe_ct> ct(new fhe_ct());
    ct->ctx = c;
    ct->level = lv;
    ct->n_poly = 2;
    ct->scale = pt->scale;
    FHE_TRY(dev_alloc(c, (void **)&ct->d, (size_t)2 * nl * N * 8));
    u64 *c0 = ct->d, *c1 = ct->d + (size_t)nl * N;
    long long *e;
    if (dev_alloc(c, (void **)&e, N * 8) != FHE_OK) {
        dev_free(ct->d);
        return FHE_E_OOM;
    }
    FHE_CU(launch_sample_uniform(c->dc, seed, DOM_ENC_A, 0, 0, 1, c1, nl, pidx.data(), 0));
    FHE_CU(launch_sample_small(c->dc, seed, DOM_ENC_E, 0, 0, 1, e, 0));
    FHE_CU(launch_signed_to_limbs(c->dc, e, c0, nl, pidx.data(), 0));
    FHE_TRY(op_ntt(c, c0, c0, 0, 1, nl, nullptr, false, 0));
    FHE_CU(launch_add(c->dc, c0, 0, pt->d, 0, c0, 0, 1, 1, lv, 0, 0));
    FHE_CU(launch_mul_limbs(c->dc, c1, sk->s_ntt, c0, 1, c0, nl, pidx.data(), 0));
    FHE_CU(cudaDeviceSynchronize());
    dev_free(e);
    *out = ct.release();
    return FHE_OK;
}

extern "C" int fhe_decrypt(fhe_ctx *c, const fhe_sk *sk, const fhe_ct *ct, fhe_pt **out) {
    if (!c || !sk || !ct || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (ct->n_poly != 2) return fhe_fail(FHE_E_INVAL, "decrypt needs a 2-polynomial ciphertext");
    FHE_CU(cudaSetDevice(c->dev));
    std::unique_ptr<fhe_pt> pt(new fhe_pt());
    pt->ctx = c;
    pt->level = ct->level;
    pt->scale = ct->scale;
    FHE_TRY(dev_alloc(c, (void **)&pt->d, (size_t)(ct->level + 1) * c->N * 8));
    FHE_CU(launch_decrypt(c->dc, ct->d, sk->s_ntt, pt->d, ct->level, 0));
    FHE_CU(cudaDeviceSynchronize());
    *out = pt.release();
    return FHE_OK;
}

// centred CRT value of residues r[0..l] as a long double (Garner's mixed radix)
static long double crt_centered(const u64 *r, int nl, const u64 *q, const std::vector<std::vector<u64>> &inv) {
    u64 v[FHE_MAX_LIMBS], w[FHE_MAX_LIMBS];
    for (int pass = 0; pass < 2; pass++) {
        u64 *d = pass == 0 ? v : w;
        for (int k = 0; k < nl; k++) {
            const u64 qk = q[k];
            u64 rk = pass == 0 ? r[k] % qk : (qk - r[k] % qk) % qk;
            u64 acc = 0;
            for (int m = k - 1; m >= 0; m--) acc = (u64)(((u128)acc * (q[m] % qk) + d[m]) % qk);
            d[k] = h_mulmod((rk + qk - acc) % qk, inv[k][0], qk);
        }
    }
    // compare x and Q - x from the most significant digit
    bool neg = false;
    for (int k = nl - 1; k >= 0; k--) {
        if (v[k] != w[k]) {
            neg = v[k] > w[k];
            break;
        }
    }
    const u64 *d = neg ? w : v;
    long double x = 0;
    for (int k = nl - 1; k >= 0; k--) x = x * (long double)q[k] + (long double)d[k];
    return neg ? -x : x;
}

extern "C" int fhe_decode(fhe_ctx *c, const fhe_pt *pt, double *re, double *im, size_t n) {
    if (!c || !pt || (n && !re)) return fhe_fail(FHE_E_INVAL, "null argument");
    if (n > (size_t)c->N / 2) return fhe_fail(FHE_E_INVAL, "more slots than N/2");
    FHE_CU(cudaSetDevice(c->dev));
    const int nl = pt->level + 1;
    const long long N = c->N;
    u64 *tmp;
    FHE_TRY(dev_alloc(c, (void **)&tmp, (size_t)nl * N * 8));
    FHE_TRY(op_ntt(c, pt->d, tmp, 0, 1, nl, nullptr, true, 0));
    std::vector<u64> h((size_t)nl * N);
    FHE_CU(cudaMemcpy(h.data(), tmp, h.size() * 8, cudaMemcpyDeviceToHost));
    dev_free(tmp);
    std::vector<std::vector<u64>> inv(nl, std::vector<u64>(1));
    for (int k = 0; k < nl; k++) {
        u64 p = 1;
        for (int m = 0; m < k; m++) p = h_mulmod(p, c->primes[m] % c->primes[k], c->primes[k]);
        inv[k][0] = h_invmod(p, c->primes[k]);
    }
    std::vector<double> m(N);
    std::vector<u64> r(nl);
    for (long long j = 0; j < N; j++) {
        for (int k = 0; k < nl; k++) r[k] = h[(size_t)k * N + j];
        m[j] = (double)crt_centered(r.data(), nl, c->primes.data(), inv);
    }
    c->enc.decode(m.data(), pt->scale, re, im, n);
    return FHE_OK;
}

// ================================================================ ciphertexts

static int new_ct(fhe_ctx *c, int level, int n_poly, double scale, fhe_ct **out) {
    std::unique_ptr<fhe_ct> ct(new fhe_ct());
    ct->ctx = c;
    ct->level = level;
    ct->n_poly = n_poly;
    ct->scale = scale;
    FHE_TRY(dev_alloc(c, (void **)&ct->d, (size_t)n_poly * (level + 1) * c->N * 8));
    *out = ct.release();
    return FHE_OK;
}

extern "C" int fhe_ct_free(fhe_ct *ct) {
    if (!ct) return FHE_OK;
    cudaDeviceSynchronize();
    dev_free(ct->d);
    delete ct;
    return FHE_OK;
}

extern "C" int fhe_ct_info(const fhe_ct *ct, int *level, int *n_poly, double *scale) {
    if (!ct) return fhe_fail(FHE_E_INVAL, "null argument");
    if (level) *level = ct->level;
    if (n_poly) *n_poly = ct->n_poly;
    if (scale) *scale = ct->scale;
    return FHE_OK;
}

extern "C" int fhe_ct_export(const fhe_ct *ct, uint64_t *buf, size_t cap, int *level, double *scale, int *n_poly) {
    if (!ct || !buf) return fhe_fail(FHE_E_INVAL, "null argument");
    fhe_ctx *c = ct->ctx;
    FHE_CU(cudaSetDevice(c->dev));
    const int nl = ct->level + 1;
    const size_t words = (size_t)ct->n_poly * nl * c->N;
    if (cap < words) return fhe_fail(FHE_E_INVAL, "buffer too small");
    u64 *tmp;
    FHE_TRY(dev_alloc(c, (void **)&tmp, words * 8));
    FHE_TRY(op_ntt(c, ct->d, tmp, (long long)nl * c->N, ct->n_poly, nl, nullptr, true, 0));
    FHE_CU(cudaMemcpy(buf, tmp, words * 8, cudaMemcpyDeviceToHost));
    dev_free(tmp);
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    if (n_poly) *n_poly = ct->n_poly;
    return FHE_OK;
}

extern "C" int fhe_ct_import(fhe_ctx *c, const uint64_t *buf, int n_poly, int level, double scale, fhe_ct **out) {
    if (!c || !buf || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (level < 0 || level > c->L) return fhe_fail(FHE_E_LEVEL, "level out of range");
    if (n_poly < 1 || n_poly > 3) return fhe_fail(FHE_E_INVAL, "n_poly must be 1..3");
    FHE_CU(cudaSetDevice(c->dev));
    const int nl = level + 1;
    const size_t words = (size_t)n_poly * nl * c->N;
    for (int p = 0; p < n_poly; p++)
        for (int l = 0; l < nl; l++) {
            const u64 *x = (const u64 *)buf + ((size_t)p * nl + l) * c->N;
            const u64 q = c->primes[l];
            for (long long j = 0; j < c->N; j++)
                if (x[j] >= q) return fhe_fail(FHE_E_INVAL, "residue out of range");
        }
    fhe_ct *ct;
    FHE_TRY(new_ct(c, level, n_poly, scale, &ct));
    cudaError_t e = cudaMemcpy(ct->d, buf, words * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fhe_ct_free(ct);
        return fhe_fail(FHE_E_CUDA, cudaGetErrorString(e));
    }
    int r = op_ntt(c, ct->d, ct->d, (long long)nl * c->N, n_poly, nl, nullptr, false, 0);
    if (r != FHE_OK) {
        fhe_ct_free(ct);
        return r;
    }
    FHE_CU(cudaDeviceSynchronize());
    *out = ct;
    return FHE_OK;
}

// ================================================================ primitives

extern "C" int fhe_rotate(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *in, int step, fhe_ct **out, void *stream) {
    if (!c || !evk || !in || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (in->n_poly != 2) return fhe_fail(FHE_E_INVAL, "rotate needs a 2-polynomial ciphertext");
    FHE_CU(cudaSetDevice(c->dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int k = galois_of_step(c, step);
    const int nl = in->level + 1;
    const long long N = c->N;
    fhe_ct *o;
    FHE_TRY(new_ct(c, in->level, 2, in->scale, &o));
    if (k == 1) {
        cudaError_t e = cudaMemcpyAsync(o->d, in->d, (size_t)2 * nl * N * 8, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            fhe_ct_free(o);
            return fhe_fail(FHE_E_CUDA, cudaGetErrorString(e));
        }
        *out = o;
        return FHE_OK;
    }
    auto it = evk->galois.find(k);
    if (it == evk->galois.end()) {
        fhe_ct_free(o);
        return fhe_fail(FHE_E_NOKEY, "no Galois key for rotation step " + std::to_string(step));
    }
    KsArgs a;
    memset(&a, 0, sizeof(a));
    a.d = in->d + (size_t)nl * N;
    a.galois = k;
    a.key = it->second;
    a.key_digits_top = evk->digits;
    a.add0 = in->d;
    a.out = o->d;
    a.n_items = 1;
    a.level = in->level;
    int r = op_keyswitch(c, a, s);
    if (r != FHE_OK) {
        fhe_ct_free(o);
        return r;
    }
    *out = o;
    return FHE_OK;
}

extern "C" int fhe_square(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *in, fhe_ct **out, void *stream) {
    if (!c || !evk || !in || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (in->n_poly != 2) return fhe_fail(FHE_E_INVAL, "square needs a 2-polynomial ciphertext");
    FHE_CU(cudaSetDevice(c->dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int nl = in->level + 1;
    const long long N = c->N;
    u64 *t3;
    FHE_ALLOC_ASYNC(&t3, (size_t)3 * nl * N * 8, s);
    FHE_CU(launch_square_act(c->dc, in->d, 0, nullptr, nullptr, t3, 0, 1, in->level, s));
    fhe_ct *o;
    FHE_TRY(new_ct(c, in->level, 2, in->scale * in->scale, &o));
    KsArgs a;
    memset(&a, 0, sizeof(a));
    a.d = t3 + (size_t)2 * nl * N;
    a.galois = 1;
    a.key = evk->relin;
    a.key_digits_top = evk->digits;
    a.add0 = t3;
    a.add1 = t3 + (size_t)nl * N;
    a.out = o->d;
    a.n_items = 1;
    a.level = in->level;
    int r = op_keyswitch(c, a, s);
    cudaFreeAsync(t3, s);
    if (r != FHE_OK) {
        fhe_ct_free(o);
        return r;
    }
    *out = o;
    return FHE_OK;
}

extern "C" int fhe_rescale(fhe_ctx *c, fhe_ct *ct, void *stream) {
    if (!c || !ct) return fhe_fail(FHE_E_INVAL, "null argument");
    if (ct->level < 1) return fhe_fail(FHE_E_LEVEL, "no level left to rescale");
    FHE_CU(cudaSetDevice(c->dev));
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = c->N;
    u64 *o;
    FHE_TRY(dev_alloc(c, (void **)&o, (size_t)ct->n_poly * ct->level * N * 8));
    int r = op_rescale(c, ct->d, 0, o, 0, 1, ct->n_poly, ct->level, s);
    if (r != FHE_OK) {
        dev_free(o);
        return r;
    }
    FHE_CU(cudaStreamSynchronize(s));
    dev_free(ct->d);
    ct->d = o;
    ct->scale = ct->scale / (double)c->primes[ct->level];
    ct->level -= 1;
    return FHE_OK;
}

extern "C" int fhe_add(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out, void *stream) {
    if (!c || !a || !b || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (a->level != b->level || a->n_poly != b->n_poly) return fhe_fail(FHE_E_LEVEL, "operands differ in level");
    if (std::fabs(a->scale - b->scale) > 1e-9 * std::fmax(std::fabs(a->scale), std::fabs(b->scale)))
        return fhe_fail(FHE_E_LEVEL, "operands differ in scale");
    FHE_CU(cudaSetDevice(c->dev));
    fhe_ct *o;
    FHE_TRY(new_ct(c, a->level, a->n_poly, a->scale, &o));
    FHE_CU(launch_add(c->dc, a->d, 0, b->d, 0, o->d, 0, 1, a->n_poly, a->level, 0, (cudaStream_t)stream));
    *out = o;
    return FHE_OK;
}

extern "C" int fhe_mul_plain(fhe_ctx *c, const fhe_ct *a, const fhe_pt *pt, fhe_ct **out, void *stream) {
    if (!c || !a || !pt || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (pt->level < a->level) return fhe_fail(FHE_E_LEVEL, "plaintext level below ciphertext level");
    FHE_CU(cudaSetDevice(c->dev));
    const int nl = a->level + 1;
    std::vector<unsigned char> pidx(nl);
    for (int t = 0; t < nl; t++) pidx[t] = (unsigned char)t;
    fhe_ct *o;
    FHE_TRY(new_ct(c, a->level, a->n_poly, a->scale * pt->scale, &o));
    for (int p = 0; p < a->n_poly; p++)
        FHE_CU(launch_mul_limbs(c->dc, a->d + (size_t)p * nl * c->N, pt->d, nullptr, 0, o->d + (size_t)p * nl * c->N,
                                nl, pidx.data(), (cudaStream_t)stream));
    *out = o;
    return FHE_OK;
}

// ================================================================ test hooks

extern "C" int fhe_ntt_device(fhe_ctx *c, uint64_t *d, size_t n_limbs, const int32_t *prime_idx, int inverse,
                              void *stream) {
    if (!c || !d || !prime_idx || n_limbs == 0) return fhe_fail(FHE_E_INVAL, "null argument");
    FHE_CU(cudaSetDevice(c->dev));
    std::vector<unsigned char> p(FHE_MAX_LIMBS);
    for (size_t off = 0; off < n_limbs; off += FHE_MAX_LIMBS) {
        const int cnt = (int)std::min<size_t>(FHE_MAX_LIMBS, n_limbs - off);
        for (int l = 0; l < cnt; l++) {
            if (prime_idx[off + l] < 0 || prime_idx[off + l] >= c->n_primes)
                return fhe_fail(FHE_E_INVAL, "prime index out of range");
            p[l] = (unsigned char)prime_idx[off + l];
        }
        u64 *dd = (u64 *)d + off * c->N;
        FHE_TRY(op_ntt(c, dd, dd, 0, 1, cnt, p.data(), inverse != 0, (cudaStream_t)stream));
    }
    return FHE_OK;
}

extern "C" int fhe_evk_export(const fhe_evk *evk, int galois, uint64_t *buf, size_t cap, size_t *n_words) {
    if (!evk || !n_words) return fhe_fail(FHE_E_INVAL, "null argument");
    fhe_ctx *c = evk->ctx;
    const u64 *k = nullptr;
    if (galois == 0) {
        k = evk->relin;
    } else {
        auto it = evk->galois.find(galois);
        if (it == evk->galois.end()) return fhe_fail(FHE_E_NOKEY, "no such Galois key");
        k = it->second;
    }
    *n_words = key_words(c);
    if (buf) {
        if (cap < *n_words) return fhe_fail(FHE_E_INVAL, "buffer too small");
        FHE_CU(cudaMemcpy(buf, k, *n_words * 8, cudaMemcpyDeviceToHost));
    }
    return FHE_OK;
}

extern "C" int fhe_profile_keyswitch(fhe_ctx *c, const fhe_evk *evk, int level, int n_items, int iters,
                                     float *ms_out, void *stream) {
    if (!c || !evk || !ms_out || n_items < 1 || iters < 1) return fhe_fail(FHE_E_INVAL, "bad argument");
    if (level < 0 || level > c->L) return fhe_fail(FHE_E_LEVEL, "level out of range");
    FHE_CU(cudaSetDevice(c->dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int nl = level + 1;
    const long long N = c->N;
    const size_t item = (size_t)3 * nl * N;   // d, then 2 output polys
    u64 *buf;
    FHE_TRY(dev_alloc(c, (void **)&buf, item * n_items * 8));
    std::vector<unsigned char> pidx(nl);
    for (int t = 0; t < nl; t++) pidx[t] = (unsigned char)t;
    for (int i = 0; i < n_items; i++)
        FHE_CU(launch_sample_uniform(c->dc, 99, 9, (uint32_t)i, 0, 1, buf + i * item, nl, pidx.data(), s));
    KsArgs a;
    memset(&a, 0, sizeof(a));
    a.d = buf;
    a.d_item = (long long)item;
    a.galois = 1;
    a.key = evk->relin;
    a.key_digits_top = evk->digits;
    a.out = buf + (size_t)nl * N;
    a.out_item = (long long)item;
    a.n_items = n_items;
    a.level = level;
    const size_t per = ks_workspace_words(c->dc, level);
    FHE_TRY(ws_reserve(c, &c->ks_ws, &c->ks_ws_words, per * (size_t)n_items));
    a.ws = c->ks_ws;
    a.ws_item = (long long)per;
    cudaEvent_t ev[9];
    for (auto &e : ev) FHE_CU(cudaEventCreate(&e));
    double acc[8] = {0};
    FHE_CU(launch_keyswitch(c->dc, c->lt[level], a, s, nullptr));   // warm-up
    for (int it = 0; it < iters; it++) {
        FHE_CU(launch_keyswitch(c->dc, c->lt[level], a, s, ev));
        FHE_CU(cudaEventSynchronize(ev[8]));
        for (int k = 0; k < 8; k++) {
            float ms;
            FHE_CU(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            acc[k] += ms;
        }
    }
    for (int k = 0; k < 8; k++) ms_out[k] = (float)(acc[k] / iters);
    for (auto &e : ev) cudaEventDestroy(e);
    dev_free(buf);
    return FHE_OK;
}

extern "C" int fhe_sk_export(const fhe_sk *sk, uint64_t *buf, size_t cap) {
    if (!sk || !buf) return fhe_fail(FHE_E_INVAL, "null argument");
    const size_t w = (size_t)sk->ctx->n_primes * sk->ctx->N;
    if (cap < w) return fhe_fail(FHE_E_INVAL, "buffer too small");
    FHE_CU(cudaMemcpy(buf, sk->s_ntt, w * 8, cudaMemcpyDeviceToHost));
    return FHE_OK;
}
