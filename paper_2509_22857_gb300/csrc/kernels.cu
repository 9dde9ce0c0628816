// RNS-CKKS hot-path kernels for sm_103a.
//
// NTT: the negacyclic transform A[j] = a(psi^(2 brv(j) + 1)) (bit-reversed
// evaluation order) is done in two passes over HBM.  With N = R1 * R2, the
// first log2(R1) Cooley-Tukey stages only mix elements that are congruent
// mod R2 ("columns" of length R1, stride R2), the remaining log2(R2) stages
// only mix contiguous "rows" of length R2.  A pass keeps 16 elements per
// thread in registers: four stages on elements strided by R/16 ("layout A"),
// one exchange through shared memory, the remaining stages on 16 contiguous
// elements ("layout B").  Butterflies are Harvey's lazy ones (values in
// [0, 4q) forward, [0, 2q) inverse) with Shoup twiddles.  The key-switching
// and rescale kernels are the same passes with their neighbouring
// arithmetic (basis conversion, key inner product, P^-1 / q_l^-1 scaling,
// Galois gathers) fused into the loads and stores.
#include "kernels.h"

#include <algorithm>
#include <atomic>
#include <cstring>

#define NT 256

// number of kernel launches issued by this library (for launch accounting)
static std::atomic<unsigned long long> g_launches{0};
unsigned long long fhe_launch_counter() { return g_launches.load(); }
void fhe_launch_counter_add(long long n) { g_launches.fetch_add((unsigned long long)n); }
#define COUNT_LAUNCH() g_launches.fetch_add(1, std::memory_order_relaxed)

namespace {

// Forward butterfly without Harvey's per-stage correction: t = w*Y mod q lies
// in [0, 2q) for any 64-bit Y, so X + t and X - t + 2q grow by at most 2q per
// stage.  Inputs below q stay below 17q after the 8 stages of one pass and
// below 33q < 2^64 (q < 2^58) after both; the second pass reduces once.
__device__ __forceinline__ void ct_bf(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    const u64 t = mul_shoup_lazy(Y, w.x, w.y, q);
    const u64 x = X;
    X = x + t;
    Y = x - t + 2 * q;
}

// full reduction of a lazy forward-NTT output (< 33q < 2^64)
__device__ __forceinline__ u64 reduce_fwd(u64 x, const ModQ &m) { return barrett(U128{x, 0}, m); }

__device__ __forceinline__ void gs_bf(u64 &X, u64 &Y, ulonglong2 w, u64 q) {
    const u64 two_q = 2 * q;
    u64 s = X + Y;
    if (s >= two_q) s -= two_q;
    u64 t = X - Y + two_q;
    X = s;
    Y = mul_shoup_lazy(t, w.x, w.y, q);
}


// Galois gather in the NTT domain: sigma_k(a) at slot j is a at slot
// brv(((2 brv(j) + 1) k mod 2N - 1) / 2).
__device__ __forceinline__ int galois_src(int j, int k, int logN) {
    if (k <= 1) return j;
    const unsigned mask2n = (2u << logN) - 1u;
    unsigned e = 2u * (__brev((unsigned)j) >> (32 - logN)) + 1u;
    unsigned ek = (unsigned)(((unsigned long long)e * (unsigned)k) & mask2n);
    return (int)(__brev((ek - 1u) >> 1) >> (32 - logN));
}

template <int LOGR>
struct Geo {
    static constexpr int R = 1 << LOGR;
    static constexpr int S = R / 16;      // threads per sub-transform
    static constexpr int T = NT / S;      // sub-transforms per CTA
    static constexpr int RP = R + R / 16; // padded row (row passes)
};

// ---- twiddle sources: entry (1 << sg) + (j >> (logN - sg)) of a table
struct TwGlobal {
    const ulonglong2 *__restrict__ t;
    int logN;
    __device__ __forceinline__ ulonglong2 operator()(int sg, int j) const {
        return __ldg(&t[(1 << sg) + (j >> (logN - sg))]);
    }
};
// column passes only touch entries below 2^logR1: staged in shared memory
struct TwShared {
    const ulonglong2 *t;
    int logN;
    __device__ __forceinline__ ulonglong2 operator()(int sg, int j) const { return t[(1 << sg) + (j >> (logN - sg))]; }
};

// ---- stages.  jb + e*js is the global index of local element e.  In every
// stage the butterflies of a group of 2*half consecutive registers share one
// twiddle, which is loaded once per group.  Each stage is its own template
// instance so that every register index is a compile-time constant (the
// 16-element tile then stays in registers instead of local memory).
// Layout A: stages s = 0..3 on elements strided by S; layout B: stages
// s = 4..LOGR-1 on 16 contiguous elements.
template <int LOGR, int s>
struct StageGeo {
    static constexpr int half = s < 4 ? (8 >> s) : ((1 << LOGR) >> (s + 1));
    // local index of the first element of the group that starts at register k0
    __device__ static __forceinline__ int elem(int tau, int k0) {
        return s < 4 ? tau + Geo<LOGR>::S * k0 : 16 * tau + k0;
    }
};

template <int LOGR, int s, class TW>
__device__ __forceinline__ void fwd_stage(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    using G = StageGeo<LOGR, s>;
#pragma unroll
    for (int k0 = 0; k0 < 16; k0 += 2 * G::half) {
        const ulonglong2 w = tw(sg0 + s, jb + G::elem(tau, k0) * js);
#pragma unroll
        for (int u = 0; u < G::half; u++) ct_bf(x[k0 + u], x[k0 + u + G::half], w, q);
    }
}

template <int LOGR, int s, class TW>
__device__ __forceinline__ void inv_stage(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    using G = StageGeo<LOGR, s>;
#pragma unroll
    for (int k0 = 0; k0 < 16; k0 += 2 * G::half) {
        const ulonglong2 w = tw(sg0 + s, jb + G::elem(tau, k0) * js);
#pragma unroll
        for (int u = 0; u < G::half; u++) gs_bf(x[k0 + u], x[k0 + u + G::half], w, q);
    }
}

template <int LOGR, class TW>
__device__ __forceinline__ void fwd_A(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    fwd_stage<LOGR, 0>(x, tau, jb, js, sg0, tw, q);
    fwd_stage<LOGR, 1>(x, tau, jb, js, sg0, tw, q);
    fwd_stage<LOGR, 2>(x, tau, jb, js, sg0, tw, q);
    fwd_stage<LOGR, 3>(x, tau, jb, js, sg0, tw, q);
}

template <int LOGR, class TW>
__device__ __forceinline__ void fwd_B(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    if constexpr (LOGR > 4) fwd_stage<LOGR, 4>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 5) fwd_stage<LOGR, 5>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 6) fwd_stage<LOGR, 6>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 7) fwd_stage<LOGR, 7>(x, tau, jb, js, sg0, tw, q);
}

template <int LOGR, class TW>
__device__ __forceinline__ void inv_B(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    if constexpr (LOGR > 7) inv_stage<LOGR, 7>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 6) inv_stage<LOGR, 6>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 5) inv_stage<LOGR, 5>(x, tau, jb, js, sg0, tw, q);
    if constexpr (LOGR > 4) inv_stage<LOGR, 4>(x, tau, jb, js, sg0, tw, q);
}

template <int LOGR, class TW>
__device__ __forceinline__ void inv_A(u64 (&x)[16], int tau, int jb, int js, int sg0, TW tw, u64 q) {
    inv_stage<LOGR, 3>(x, tau, jb, js, sg0, tw, q);
    inv_stage<LOGR, 2>(x, tau, jb, js, sg0, tw, q);
    inv_stage<LOGR, 1>(x, tau, jb, js, sg0, tw, q);
    inv_stage<LOGR, 0>(x, tau, jb, js, sg0, tw, q);
}

// stage the first 2^LOGR twiddles (all a column pass uses) in shared memory
template <int LOGR>
__device__ __forceinline__ TwShared stage_twiddles(ulonglong2 *sm_tw, const ulonglong2 *__restrict__ tab, int logN) {
    for (int i = threadIdx.x; i < (1 << LOGR); i += NT) sm_tw[i] = __ldg(&tab[i]);
    __syncthreads();
    return TwShared{sm_tw, logN};
}

// ---- exchanges through shared memory
// column passes: sm[e*T + cl]
template <int LOGR>
__device__ __forceinline__ void xchg_col_AB(u64 (&x)[16], u64 *sm, int tau, int cl) {
    constexpr int S = Geo<LOGR>::S, T = Geo<LOGR>::T;
#pragma unroll
    for (int k = 0; k < 16; k++) sm[(tau + S * k) * T + cl] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[(16 * tau + k) * T + cl];
    __syncthreads();
}
template <int LOGR>
__device__ __forceinline__ void xchg_col_BA(u64 (&x)[16], u64 *sm, int tau, int cl) {
    constexpr int S = Geo<LOGR>::S, T = Geo<LOGR>::T;
#pragma unroll
    for (int k = 0; k < 16; k++) sm[(16 * tau + k) * T + cl] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[(tau + S * k) * T + cl];
    __syncthreads();
}
// row passes: sm[rl*RP + e + e/16]
template <int LOGR>
__device__ __forceinline__ void xchg_row_AB(u64 (&x)[16], u64 *sm, int tau, int rl) {
    constexpr int S = Geo<LOGR>::S, RP = Geo<LOGR>::RP;
    u64 *r = sm + rl * RP;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = tau + S * k;
        r[e + (e >> 4)] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = 16 * tau + k;
        x[k] = r[e + (e >> 4)];
    }
    __syncthreads();
}
template <int LOGR>
__device__ __forceinline__ void xchg_row_BA(u64 (&x)[16], u64 *sm, int tau, int rl) {
    constexpr int S = Geo<LOGR>::S, RP = Geo<LOGR>::RP;
    u64 *r = sm + rl * RP;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = 16 * tau + k;
        r[e + (e >> 4)] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = tau + S * k;
        x[k] = r[e + (e >> 4)];
    }
    __syncthreads();
}

constexpr int SMEM_WORDS = 4096 + 256;
// elements per thread whose basis-conversion sums are accumulated together,
// and the conversion kernels' blocks per SM (register bound)
#ifndef CONV_CHUNK
#define CONV_CHUNK 4
#endif
#ifndef CONV_MINB
#define CONV_MINB 3
#endif

// ================================================================ plain NTT

// forward pass 1 (columns of length 2^LOGR = 2^logR1)
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ntt_fwd_col(DevCtx c, NttArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y, item = job / a.n_limbs, limb = job % a.n_limbs;
    const PrimeTab &P = c.primes[a.pidx[limb]];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.fwd, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    const u64 *src = a.src + item * a.src_item + ((long long)limb << c.logN);
    u64 *dst = a.dst + item * a.dst_item + ((long long)limb << c.logN);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = src[col + ((tau + Gm::S * k) << logC)];
    fwd_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_AB<LOGR>(x, sm, tau, cl);
    fwd_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) dst[col + ((16 * tau + k) << logC)] = x[k];
}

// forward pass 2 (rows of length 2^LOGR = 2^logR2), in place on dst
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ntt_fwd_row(DevCtx c, NttArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y, item = job / a.n_limbs, limb = job % a.n_limbs;
    const PrimeTab &P = c.primes[a.pidx[limb]];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    u64 *p = a.dst + item * a.dst_item + ((long long)limb << c.logN) + (row << LOGR);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[tau + Gm::S * k];
    fwd_A<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    fwd_B<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
#pragma unroll
    for (int k = 0; k < 16; k++) p[tau + Gm::S * k] = reduce_fwd(x[k], P.m);
}

// inverse pass 1 (rows)
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ntt_inv_row(DevCtx c, NttArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y, item = job / a.n_limbs, limb = job % a.n_limbs;
    const PrimeTab &P = c.primes[a.pidx[limb]];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const u64 *s = a.src + item * a.src_item + ((long long)limb << c.logN) + (row << LOGR);
    u64 *d = a.dst + item * a.dst_item + ((long long)limb << c.logN) + (row << LOGR);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = s[tau + Gm::S * k];
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    inv_B<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
    inv_A<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
#pragma unroll
    for (int k = 0; k < 16; k++) d[tau + Gm::S * k] = x[k];
}

// inverse pass 2 (columns), times N^-1, in place on dst
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ntt_inv_col(DevCtx c, NttArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y, item = job / a.n_limbs, limb = job % a.n_limbs;
    const PrimeTab &P = c.primes[a.pidx[limb]];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.inv, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    u64 *p = a.dst + item * a.dst_item + ((long long)limb << c.logN);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[col + ((16 * tau + k) << logC)];
    inv_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_BA<LOGR>(x, sm, tau, cl);
    inv_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 v = mul_shoup_lazy(x[k], P.n_inv, P.n_inv_sh, q);
        p[col + ((tau + Gm::S * k) << logC)] = v >= q ? v - q : v;
    }
}

// ================================================================ key switching

struct KsLayout {
    long long y, mu, acc, z, md, u;   // word offsets inside one item's workspace
};

__host__ __device__ inline KsLayout ks_layout(int level, int n_digits, int alpha, int logN) {
    const long long N = 1ll << logN;
    const int ext = level + 1 + alpha;
    KsLayout L;
    L.y = 0;
    L.mu = L.y + (level + 1) * N;
    L.acc = L.mu + (long long)n_digits * ext * N;
    L.z = L.acc + 2ll * ext * N;
    L.md = L.z + 2ll * alpha * N;
    L.u = L.md + 2ll * (level + 1) * N;
    return L;
}

// (1) iNTT rows of d (with Galois gather) -> y region
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ks_intt_row(DevCtx c, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int nl = a.level + 1;
    const int job = blockIdx.y, item = job / nl, limb = job % nl;
    const PrimeTab &P = c.primes[limb];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const u64 *s = a.d + item * a.d_item + ((long long)limb << c.logN);
    u64 *d = a.ws + item * a.ws_item + ly.y + ((long long)limb << c.logN) + (row << LOGR);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = s[galois_src((row << LOGR) + tau + Gm::S * k, a.galois, c.logN)];
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    inv_B<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
    inv_A<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
#pragma unroll
    for (int k = 0; k < 16; k++) d[tau + Gm::S * k] = x[k];
}

// (2) iNTT columns, times N^-1 * Qhat_{j,i}^-1 -> y
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ks_intt_col(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int nl = a.level + 1;
    const int job = blockIdx.y, item = job / nl, limb = job % nl;
    const PrimeTab &P = c.primes[limb];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.inv, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    u64 *p = a.ws + item * a.ws_item + ly.y + ((long long)limb << c.logN);
    const ulonglong2 sc = lt.y_scale[limb];
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[col + ((16 * tau + k) << logC)];
    inv_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_BA<LOGR>(x, sm, tau, cl);
    inv_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 v = mul_shoup_lazy(x[k], sc.x, sc.y, q);
        p[col + ((tau + Gm::S * k) << logC)] = v >= q ? v - q : v;
    }
}

// (3) ModUp: basis conversion of digit j to ext limb t fused with NTT columns
template <int LOGR>
__global__ void __launch_bounds__(NT, CONV_MINB) k_ks_modup_col(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int ext = lt.ext, nd = lt.n_digits;
    const int job = blockIdx.y;
    const int item = job / (nd * ext);
    const int j = (job / ext) % nd;
    const int t = job % ext;
    const int alpha = c.alpha;
    const int d_lo = j * alpha;
    const int d_hi = min(d_lo + alpha, a.level + 1);
    if (t >= d_lo && t < d_hi) return;   // limb of the digit itself: no conversion
    const PrimeTab &P = c.primes[ext_prime(t, a.level, c.L)];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.fwd, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    const u64 *y = a.ws + item * a.ws_item + ly.y;
    u64 *dst = a.ws + item * a.ws_item + ly.mu + ((long long)(j * ext + t) << c.logN);
    const u64 *hat = lt.modup_hat + (long long)(j * alpha) * ext;
    const int nu = d_hi - d_lo;
    // sum over the digit's primes: runtime loop outside, 8 elements inside
    const long long sc = (long long)Gm::S << logC;
    u64 x[16];
#pragma unroll
    for (int h8 = 0; h8 < 16; h8 += CONV_CHUNK) {
        U128 acc[CONV_CHUNK];
#pragma unroll
        for (int k = 0; k < CONV_CHUNK; k++) acc[k] = U128{0, 0};
        for (int u = 0; u < nu; u++) {
            const u64 h = hat[u * ext + t];
            const u64 *yp = y + ((long long)(d_lo + u) << c.logN) + col + ((long long)tau << logC) + h8 * sc;
            u64 v[CONV_CHUNK];
#pragma unroll
            for (int k = 0; k < CONV_CHUNK; k++) v[k] = yp[k * sc];
#pragma unroll
            for (int k = 0; k < CONV_CHUNK; k++) mac(acc[k], v[k], h);
        }
#pragma unroll
        for (int k = 0; k < CONV_CHUNK; k++) x[h8 + k] = barrett(acc[k], P.m);
    }
    fwd_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_AB<LOGR>(x, sm, tau, cl);
    fwd_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) dst[col + ((16 * tau + k) << logC)] = x[k];
}

// (4) ModUp: NTT rows of every converted limb, in place
template <int LOGR>
__global__ void __launch_bounds__(NT, 3) k_ks_modup_row(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int ext = lt.ext, nd = lt.n_digits;
    const int job = blockIdx.y;
    const int item = job / (nd * ext);
    const int j = (job / ext) % nd;
    const int t = job % ext;
    const int d_lo = j * c.alpha, d_hi = min(d_lo + c.alpha, a.level + 1);
    if (t >= d_lo && t < d_hi) return;
    const PrimeTab &P = c.primes[ext_prime(t, a.level, c.L)];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const int base = row << LOGR;
    u64 *p = a.ws + item * a.ws_item + ly.mu + ((long long)(j * ext + t) << c.logN) + base;
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[tau + Gm::S * k];
    fwd_A<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    fwd_B<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
#pragma unroll
    for (int k = 0; k < 16; k++) p[tau + Gm::S * k] = reduce_fwd(x[k], P.m);
}

// (4b) inner product with the key, acc_k[t] = sum_j ext_j[t] * key_j[k][t],
// for ND digits.  Each thread takes two adjacent NTT slots and loops over
// the items of the batch, so each key coefficient is fetched from HBM once
// per batch.
// In the bit-reversed NTT order a Galois gather maps every aligned pair of
// slots onto an aligned pair (in swapped order when the source index is odd),
// so each operand pair is one 16-byte load.  ND sizes the key and operand
// registers exactly, which keeps more loads in flight per SM than the scalar
// kernel with one slot per thread and arrays for 7 digits, which was latency-bound.
__device__ __forceinline__ ulonglong2 ld_pair(const u64 *p, bool swap) {
    ulonglong2 v = *(const ulonglong2 *)p;
    return swap ? make_ulonglong2(v.y, v.x) : v;
}

// double hoisting: poly 0 of a rotation kept in Q_l u P is the inner product
// plus P sigma(c0); on Q limb t that adds (P mod q_t) c0 at the gathered slot
__device__ __forceinline__ ulonglong2 ip_fold_pair(const DevCtx &c, const KsArgs &a, int item, int t, int ip_col,
                                                   bool ip_sw, ulonglong2 r0, const ModQ &m) {
    const long long N = 1ll << c.logN;
    const ulonglong2 f = ld_pair(a.ip_fold + item * a.ip_fold_item + (long long)t * N + (ip_col & ~1), ip_sw);
    const u64 pm = c.md_pmod[t];
    return make_ulonglong2(add_mod(r0.x, mulmod(f.x, pm, m), m.q), add_mod(r0.y, mulmod(f.y, pm, m), m.q));
}

// XO: the double-hoisting form (ip_out / ip_fold honoured); the plain form
// is its own instance, so its code is not burdened by the extra paths
template <int ND, bool XO>
__global__ void __launch_bounds__(256) k_ks_ip(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    const int ext = lt.ext;
    const int t = blockIdx.y;
    const int pi = ext_prime(t, a.level, c.L);
    const ModQ m = c.primes[pi].m;
    const long long N = 1ll << c.logN;
    const int col = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const long long key_limbs = c.L + 1 + c.alpha;
    const int jt = t <= a.level ? t / c.alpha : -1;   // digit that holds limb t itself
    const int ip_col = galois_src(col, a.ip_galois, c.logN);
    const int src_col = jt >= 0 ? galois_src(ip_col, a.galois, c.logN) : ip_col;
    const bool ip_sw = ip_col & 1, src_sw = src_col & 1;
    ulonglong2 k0[ND], k1[ND];
#pragma unroll
    for (int j = 0; j < ND; j++) {
        const u64 *kb = a.key + ((long long)(j * 2) * key_limbs + pi) * N + col;
        k0[j] = __ldg((const ulonglong2 *)kb);
        k1[j] = __ldg((const ulonglong2 *)(kb + key_limbs * N));
    }
    for (int item = 0; item < a.n_items; item++) {
        const u64 *mu = a.ws + item * a.ws_item + ly.mu + (long long)t * N + (ip_col & ~1);
        const u64 *dd = a.d + item * a.d_item + (long long)t * N + (src_col & ~1);
        ulonglong2 x[ND];
#pragma unroll
        for (int j = 0; j < ND; j++) x[j] = (j == jt) ? ld_pair(dd, src_sw) : ld_pair(mu + (long long)j * ext * N, ip_sw);
        U128 a00 = {0, 0}, a01 = {0, 0}, a10 = {0, 0}, a11 = {0, 0};
#pragma unroll
        for (int j = 0; j < ND; j++) {
            mac(a00, x[j].x, k0[j].x);
            mac(a01, x[j].y, k0[j].y);
            mac(a10, x[j].x, k1[j].x);
            mac(a11, x[j].y, k1[j].y);
        }
        u64 *ob = XO && a.ip_out ? a.ip_out + item * a.ip_out_item : a.ws + item * a.ws_item + ly.acc;
        ulonglong2 *o0 = (ulonglong2 *)(ob + (long long)t * N + col);
        ulonglong2 *o1 = (ulonglong2 *)((u64 *)o0 + (long long)ext * N);
        ulonglong2 r0 = make_ulonglong2(barrett(a00, m), barrett(a01, m));
        ulonglong2 r1 = make_ulonglong2(barrett(a10, m), barrett(a11, m));
        if (XO && a.ip_fold && t <= a.level) r0 = ip_fold_pair(c, a, item, t, ip_col, ip_sw, r0, m);
        if (a.ip_accumulate) {
            const ulonglong2 p0 = *o0, p1 = *o1;
            r0 = make_ulonglong2(add_mod(r0.x, p0.x, m.q), add_mod(r0.y, p0.y, m.q));
            r1 = make_ulonglong2(add_mod(r1.x, p1.x, m.q), add_mod(r1.y, p1.y, m.q));
        }
        *o0 = r0;
        *o1 = r1;
    }
}

template <int ND>
__global__ void __launch_bounds__(256) k_ks_ip_babies(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly, IpBabies bb) {
    const int ext = lt.ext;
    const int t = blockIdx.y;
    const int pi = ext_prime(t, a.level, c.L);
    const ModQ m = c.primes[pi].m;
    const long long N = 1ll << c.logN;
    const int col = 2 * (blockIdx.x * blockDim.x + threadIdx.x);   // source slots col, col + 1
    const long long key_limbs = c.L + 1 + c.alpha;
    const int jt = t <= a.level ? t / c.alpha : -1;   // digit that holds limb t itself
    const bool fold = a.ip_fold && t <= a.level;
    const u64 pm = fold ? c.md_pmod[t] : 0;
    for (int item = 0; item < a.n_items; item++) {
        const u64 *mu = a.ws + item * a.ws_item + ly.mu + (long long)t * N + col;
        const u64 *dd = a.d + item * a.d_item + (long long)t * N + col;
        ulonglong2 x[ND];
#pragma unroll
        for (int j = 0; j < ND; j++)
            x[j] = (j == jt) ? *(const ulonglong2 *)dd : *(const ulonglong2 *)(mu + (long long)j * ext * N);
        const ulonglong2 f =
            fold ? *(const ulonglong2 *)(a.ip_fold + item * a.ip_fold_item + (long long)t * N + col)
                 : make_ulonglong2(0, 0);
        for (int k = 0; k < bb.n; k++) {
            // the output slots fed by source slots col, col + 1: an aligned
            // pair, swapped when the first is odd
            const int jo = galois_src(col, bb.gal_inv[k], c.logN);
            const bool sw = jo & 1;
            const long long jb = jo & ~1;
            U128 a00 = {0, 0}, a01 = {0, 0}, a10 = {0, 0}, a11 = {0, 0};
#pragma unroll
            for (int j = 0; j < ND; j++) {
                const u64 *kb = bb.key[k] + ((long long)(j * 2) * key_limbs + pi) * N + jb;
                const ulonglong2 k0 = ld_pair(kb, sw);
                const ulonglong2 k1 = ld_pair(kb + key_limbs * N, sw);
                mac(a00, x[j].x, k0.x);
                mac(a01, x[j].y, k0.y);
                mac(a10, x[j].x, k1.x);
                mac(a11, x[j].y, k1.y);
            }
            ulonglong2 r0 = make_ulonglong2(barrett(a00, m), barrett(a01, m));
            const ulonglong2 r1 = make_ulonglong2(barrett(a10, m), barrett(a11, m));
            if (fold)
                r0 = make_ulonglong2(add_mod(r0.x, mulmod(f.x, pm, m), m.q), add_mod(r0.y, mulmod(f.y, pm, m), m.q));
            u64 *ob = bb.out[k] + item * a.ip_out_item + (long long)t * N + jb;
            *(ulonglong2 *)ob = sw ? make_ulonglong2(r0.y, r0.x) : r0;
            *(ulonglong2 *)(ob + (long long)ext * N) = sw ? make_ulonglong2(r1.y, r1.x) : r1;
        }
    }
}

// Inner product for more than 7 digits (one special prime per digit, as in
// the paper's own parameter sets): the digits are a loop and the key pairs
// are loaded per item, since they no longer fit in registers.  Same layout,
// gathers and arithmetic as k_ks_ip.
__global__ void __launch_bounds__(256) k_ks_ip_n(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    const int ext = lt.ext, nd = lt.n_digits;
    const int t = blockIdx.y;
    const int pi = ext_prime(t, a.level, c.L);
    const ModQ m = c.primes[pi].m;
    const long long N = 1ll << c.logN;
    const int col = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const long long key_limbs = c.L + 1 + c.alpha;
    const int jt = t <= a.level ? t / c.alpha : -1;
    const int ip_col = galois_src(col, a.ip_galois, c.logN);
    const int src_col = jt >= 0 ? galois_src(ip_col, a.galois, c.logN) : ip_col;
    const bool ip_sw = ip_col & 1, src_sw = src_col & 1;
    for (int item = 0; item < a.n_items; item++) {
        const u64 *mu = a.ws + item * a.ws_item + ly.mu + (long long)t * N + (ip_col & ~1);
        const u64 *dd = a.d + item * a.d_item + (long long)t * N + (src_col & ~1);
        U128 a00 = {0, 0}, a01 = {0, 0}, a10 = {0, 0}, a11 = {0, 0};
        for (int j = 0; j < nd; j++) {
            const ulonglong2 x = (j == jt) ? ld_pair(dd, src_sw) : ld_pair(mu + (long long)j * ext * N, ip_sw);
            const u64 *kb = a.key + ((long long)(j * 2) * key_limbs + pi) * N + col;
            const ulonglong2 k0 = __ldg((const ulonglong2 *)kb);
            const ulonglong2 k1 = __ldg((const ulonglong2 *)(kb + key_limbs * N));
            mac(a00, x.x, k0.x);
            mac(a01, x.y, k0.y);
            mac(a10, x.x, k1.x);
            mac(a11, x.y, k1.y);
        }
        u64 *ob = a.ip_out ? a.ip_out + item * a.ip_out_item : a.ws + item * a.ws_item + ly.acc;
        ulonglong2 *o0 = (ulonglong2 *)(ob + (long long)t * N + col);
        ulonglong2 *o1 = (ulonglong2 *)((u64 *)o0 + (long long)ext * N);
        ulonglong2 r0 = make_ulonglong2(barrett(a00, m), barrett(a01, m));
        ulonglong2 r1 = make_ulonglong2(barrett(a10, m), barrett(a11, m));
        if (a.ip_fold && t <= a.level) r0 = ip_fold_pair(c, a, item, t, ip_col, ip_sw, r0, m);
        if (a.ip_accumulate) {
            const ulonglong2 p0 = *o0, p1 = *o1;
            r0 = make_ulonglong2(add_mod(r0.x, p0.x, m.q), add_mod(r0.y, p0.y, m.q));
            r1 = make_ulonglong2(add_mod(r1.x, p1.x, m.q), add_mod(r1.y, p1.y, m.q));
        }
        *o0 = r0;
        *o1 = r1;
    }
}

// out[i][t] (+)= in[i][t] gathered by sigma_galois, limbs 0..level
__global__ void k_gather_acc(DevCtx c, const u64 *in, long long in_item, u64 *out, long long out_item, int level,
                             int galois, int accumulate) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int limb = blockIdx.y;
    const u64 q = c.primes[limb].m.q;
    const u64 *src = in + item * in_item + (long long)limb * N;
    u64 *dst = out + item * out_item + (long long)limb * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        u64 v = src[galois_src((int)j, galois, c.logN)];
        if (accumulate) v = add_mod(v, dst[j], q);
        dst[j] = v;
    }
}

// (5) ModDown: iNTT rows of the P limbs of acc
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ks_md_intt_row(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int al = c.alpha;
    const int job = blockIdx.y, item = job / (2 * al), kk = (job / al) % 2, m = job % al;
    const PrimeTab &P = c.primes[c.L + 1 + m];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const long long N = 1ll << c.logN;
    const u64 *accb = a.md_in ? a.md_in + item * a.md_in_item : a.ws + item * a.ws_item + ly.acc;
    const u64 *s = accb + ((long long)kk * lt.ext + a.level + 1 + m) * N + (row << LOGR);
    u64 *d = a.ws + item * a.ws_item + ly.z + ((long long)kk * al + m) * N + (row << LOGR);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = s[tau + Gm::S * k];
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    inv_B<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
    inv_A<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
#pragma unroll
    for (int k = 0; k < 16; k++) d[tau + Gm::S * k] = x[k];
}

// (6) ModDown: iNTT columns; z = (v + floor(P/2)) * Phat_m^-1 mod p_m
template <int LOGR>
__global__ void __launch_bounds__(NT) k_ks_md_intt_col(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int al = c.alpha;
    const int job = blockIdx.y, item = job / (2 * al), kk = (job / al) % 2, m = job % al;
    const PrimeTab &P = c.primes[c.L + 1 + m];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.inv, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    u64 *p = a.ws + item * a.ws_item + ly.z + ((long long)(kk * al + m) << c.logN);
    const ulonglong2 sc = c.md_z_scale[m];
    const u64 add = c.md_z_add[m];
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[col + ((16 * tau + k) << logC)];
    inv_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_BA<LOGR>(x, sm, tau, cl);
    inv_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 v = mul_shoup_lazy(x[k], sc.x, sc.y, q);
        v = v >= q ? v - q : v;
        p[col + ((tau + Gm::S * k) << logC)] = add_mod(v, add, q);
    }
}

// (6b) ModDown: overshoot of the fast conversion from P, per coefficient:
// z_m = [x (P/p_m)^-1]_{p_m} for x = [acc]_P + floor(P/2) in [0, P), and
// sum_m z_m (P/p_m) = x + u P with u = floor(sum_m z_m / p_m).  The sum is
// taken in fixed point, sum_m z_m floor(2^E / p_m) < 2^(E+3) in 128 bits;
// it falls short of 2^E sum_m z_m / p_m by less than alpha 2^58, so its
// integer part is u unless x / P lies within 2^-60 of 1.
__global__ void k_ks_md_overflow(DevCtx c, KsArgs a, KsLayout ly) {
    const long long N = 1ll << c.logN;
    const int job = blockIdx.y, item = job / 2, kk = job % 2;
    const int al = c.alpha;
    const u64 *z = a.ws + item * a.ws_item + ly.z + (long long)kk * al * N;
    u64 *u = a.ws + item * a.ws_item + ly.u + (long long)kk * N;
    const int sh = c.md_E - 64;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        U128 s = {0, 0};
        for (int m = 0; m < al; m++) mac(s, z[(long long)m * N + j], __ldg(&c.md_w[m]));
        u[j] = s.hi >> sh;
    }
}

// (7) ModDown: basis conversion P -> q_i (minus floor(P/2)) fused with NTT columns
template <int LOGR>
__global__ void __launch_bounds__(NT, CONV_MINB) k_ks_md_conv_col(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int al = c.alpha;
    const int nl = a.level + 1;
    const int job = blockIdx.y, item = job / (2 * nl), kk = (job / nl) % 2, i = job % nl;
    const PrimeTab &P = c.primes[i];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.fwd, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    const long long N = 1ll << c.logN;
    const u64 *z = a.ws + item * a.ws_item + ly.z + (long long)kk * al * N;
    u64 *dst = a.ws + item * a.ws_item + ly.md + ((long long)(kk * nl + i) << c.logN);
    const u64 halfp = c.md_halfp[i];
    const u64 pmod = c.md_pmod[i];
    const u64 *uo = a.ws + item * a.ws_item + ly.u + (long long)kk * N;
    const long long sc = (long long)Gm::S << logC;
    u64 x[16];
#pragma unroll
    for (int h8 = 0; h8 < 16; h8 += CONV_CHUNK) {
        U128 acc[CONV_CHUNK];
#pragma unroll
        for (int k = 0; k < CONV_CHUNK; k++) acc[k] = U128{0, 0};
        for (int u = 0; u < al; u++) {
            const u64 h = c.md_phat[u * (c.L + 1) + i];
            const u64 *zp = z + (long long)u * N + col + ((long long)tau << logC) + h8 * sc;
            u64 v[CONV_CHUNK];
#pragma unroll
            for (int k = 0; k < CONV_CHUNK; k++) v[k] = zp[k * sc];
#pragma unroll
            for (int k = 0; k < CONV_CHUNK; k++) mac(acc[k], v[k], h);
        }
#pragma unroll
        for (int k = 0; k < CONV_CHUNK; k++) {
            // exact conversion: remove u P (u < alpha, so u * (P mod q) < 2^64)
            const u64 uP = barrett(U128{uo[col + ((long long)tau << logC) + (h8 + k) * sc] * pmod, 0}, P.m);
            x[h8 + k] = sub_mod(sub_mod(barrett(acc[k], P.m), halfp, q), uP, q);
        }
    }
    fwd_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_AB<LOGR>(x, sm, tau, cl);
    fwd_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) dst[col + ((16 * tau + k) << logC)] = x[k];
}

// (8) ModDown: NTT rows, out_k = (acc_k - conv) * P^-1 (+ addend) (+= out)
template <int LOGR>
__global__ void __launch_bounds__(NT, 3) k_ks_md_row_out(DevCtx c, LevelTab lt, KsArgs a, KsLayout ly) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int nl = a.level + 1;
    const int job = blockIdx.y, item = job / (2 * nl), kk = (job / nl) % 2, i = job % nl;
    const PrimeTab &P = c.primes[i];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const int base = row << LOGR;
    const long long N = 1ll << c.logN;
    const u64 *s = a.ws + item * a.ws_item + ly.md + (long long)(kk * nl + i) * N + base;
    const u64 *accb = a.md_in ? a.md_in + item * a.md_in_item : a.ws + item * a.ws_item + ly.acc;
    const u64 *ac = accb + ((long long)kk * lt.ext + i) * N + base;
    const u64 *addp = kk == 0 ? a.add0 : a.add1;
    const ulonglong2 pinv = c.md_pinv[i];
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = s[tau + Gm::S * k];
    fwd_A<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    fwd_B<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
    u64 *o = a.out + item * a.out_item + ((long long)kk * nl + i) * N + base;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = tau + Gm::S * k;
        u64 v = sub_mod(ac[e], reduce_fwd(x[k], P.m), q);
        v = mul_shoup(v, pinv.x, pinv.y, q);
        if (addp) {
            const u64 *ap = addp + item * a.add_item + (long long)i * N;
            v = add_mod(v, ap[galois_src(base + e, a.add_galois, c.logN)], q);
        }
        if (a.base) v = add_mod(v, a.base[item * a.base_item + ((long long)kk * nl + i) * N + base + e], q);
        o[e] = v;
    }
}

// ================================================================ rescale

template <int LOGR>
__global__ void __launch_bounds__(NT) k_rs_intt_row(DevCtx c, RescaleArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y, item = job / a.n_poly, poly = job % a.n_poly;
    const int lv = a.level;
    const PrimeTab &P = c.primes[lv];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const long long N = 1ll << c.logN;
    const u64 *s = a.in + item * a.in_item + (long long)(poly * (lv + 1) + lv) * N + (row << LOGR);
    u64 *d = a.ws + (long long)job * N + (row << LOGR);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = s[tau + Gm::S * k];
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    inv_B<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
    inv_A<LOGR>(x, tau, row << LOGR, 1, c.logR1, TwGlobal{P.inv, c.logN}, q);
#pragma unroll
    for (int k = 0; k < 16; k++) d[tau + Gm::S * k] = x[k];
}

template <int LOGR>
__global__ void __launch_bounds__(NT) k_rs_intt_col(DevCtx c, RescaleArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int job = blockIdx.y;
    const PrimeTab &P = c.primes[a.level];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.inv, c.logN);
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    u64 *p = a.ws + ((long long)job << c.logN);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[col + ((16 * tau + k) << logC)];
    inv_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_BA<LOGR>(x, sm, tau, cl);
    inv_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 v = mul_shoup_lazy(x[k], P.n_inv, P.n_inv_sh, q);
        p[col + ((tau + Gm::S * k) << logC)] = v >= q ? v - q : v;
    }
}

// centred top limb reduced mod q_i, NTT columns; written into out limb i
template <int LOGR>
__global__ void __launch_bounds__(NT) k_rs_conv_col(DevCtx c, LevelTab lt, RescaleArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int lv = a.level;
    const int job = blockIdx.y, item = job / (a.n_poly * lv), poly = (job / lv) % a.n_poly, i = job % lv;
    const PrimeTab &P = c.primes[i];
    const u64 q = P.m.q;
    __shared__ ulonglong2 sm_tw[256];
    const TwShared tws = stage_twiddles<LOGR>(sm_tw, P.fwd, c.logN);
    const u64 ql = c.primes[lv].m.q;
    const u64 qlmod = lt.q_last_mod[i];
    const int logC = c.logN - LOGR;
    const int cl = threadIdx.x % Gm::T, tau = threadIdx.x / Gm::T;
    const int col = blockIdx.x * Gm::T + cl;
    const u64 *v = a.ws + ((long long)(item * a.n_poly + poly) << c.logN);
    u64 *dst = a.out + item * a.out_item + ((long long)(poly * lv + i) << c.logN);
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const u64 t = v[col + ((tau + Gm::S * k) << logC)];
        u64 r = barrett(U128{t, 0}, P.m);
        if (t > (ql - 1) / 2) r = sub_mod(r, qlmod, q);
        x[k] = r;
    }
    fwd_A<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
    xchg_col_AB<LOGR>(x, sm, tau, cl);
    fwd_B<LOGR>(x, tau, col, 1 << logC, 0, tws, q);
#pragma unroll
    for (int k = 0; k < 16; k++) dst[col + ((16 * tau + k) << logC)] = x[k];
}

template <int LOGR>
__global__ void __launch_bounds__(NT, 3) k_rs_row_out(DevCtx c, LevelTab lt, RescaleArgs a) {
    using Gm = Geo<LOGR>;
    __shared__ u64 sm[SMEM_WORDS];
    const int lv = a.level;
    const int job = blockIdx.y, item = job / (a.n_poly * lv), poly = (job / lv) % a.n_poly, i = job % lv;
    const PrimeTab &P = c.primes[i];
    const u64 q = P.m.q;
    const int tau = threadIdx.x % Gm::S, rl = threadIdx.x / Gm::S;
    const int row = blockIdx.x * Gm::T + rl;
    const int base = row << LOGR;
    const long long N = 1ll << c.logN;
    u64 *o = a.out + item * a.out_item + (long long)(poly * lv + i) * N + base;
    const u64 *src = a.in + item * a.in_item + (long long)(poly * (lv + 1) + i) * N + base;
    const ulonglong2 inv = lt.q_last_inv[i];
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = o[tau + Gm::S * k];
    fwd_A<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_AB<LOGR>(x, sm, tau, rl);
    fwd_B<LOGR>(x, tau, base, 1, c.logR1, TwGlobal{P.fwd, c.logN}, q);
    xchg_row_BA<LOGR>(x, sm, tau, rl);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int e = tau + Gm::S * k;
        u64 v = sub_mod(src[e], reduce_fwd(x[k], P.m), q);
        o[e] = mul_shoup(v, inv.x, inv.y, q);
    }
}

// ================================================================ elementwise

__global__ void k_add(DevCtx c, const u64 *a, long long a_item, const u64 *b, long long b_item, u64 *out,
                      long long out_item, int n_poly, int level, int subtract) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int pl = blockIdx.y;  // poly * (level+1) + limb
    const int limb = pl % (level + 1);
    const u64 q = c.primes[limb].m.q;
    const long long off = (long long)pl * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        u64 x = a[item * a_item + off + j], y = b[item * b_item + off + j];
        out[item * out_item + off + j] = subtract ? sub_mod(x, y, q) : add_mod(x, y, q);
    }
}

__global__ void k_mul_const(DevCtx c, const u64 *a, long long a_item, const u64 *cst, u64 *out,
                            long long out_item, int level) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int pl = blockIdx.y;
    const int limb = pl % (level + 1);
    const ModQ m = c.primes[limb].m;
    const u64 w = cst[limb];
    const long long off = (long long)pl * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x)
        out[item * out_item + off + j] = mulmod(a[item * a_item + off + j], w, m);
}

__global__ void k_add_const(DevCtx c, const u64 *a, long long a_item, const u64 *cst, u64 *out,
                            long long out_item, int level) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int pl = blockIdx.y;  // 2*(level+1)
    const int limb = pl % (level + 1);
    const u64 q = c.primes[limb].m.q;
    const u64 w = pl < level + 1 ? cst[limb] : 0;
    const long long off = (long long)pl * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x)
        out[item * out_item + off + j] = add_mod(a[item * a_item + off + j], w, q);
}

__global__ void k_square_act(DevCtx c, const u64 *in, long long in_item, const u64 *c1, const u64 *c0,
                             u64 *out, long long out_item, int level, const u64 *c1v, const u64 *c0v, int n_ct) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int limb = blockIdx.y;
    const ModQ m = c.primes[limb].m;
    const long long P = (long long)(level + 1) * N;
    const u64 s1 = c1 ? c1[limb] : 0, s0 = c0 ? c0[limb] : 0;
    // per-channel coefficients: this ciphertext's plaintexts, limb `limb`
    const long long voff = (long long)(item % n_ct) * P + (long long)limb * N;
    const u64 *x = in + item * in_item + (long long)limb * N;
    u64 *o = out + item * out_item + (long long)limb * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const u64 w1 = c1v ? c1v[voff + j] : s1, w0 = c1v ? c0v[voff + j] : s0;
        const u64 a = x[j], b = x[P + j];
        U128 t0 = mul_wide(a, a);
        mac(t0, w1, a);
        u64 d0 = add_mod(barrett(t0, m), w0, m.q);
        U128 t1 = mul_wide(a, b);
        add_to(t1, t1);
        mac(t1, w1, b);
        o[j] = d0;
        o[P + j] = barrett(t1, m);
        o[2 * P + j] = mulmod(b, b, m);
    }
}

__global__ void k_drop(DevCtx c, const u64 *in, long long in_item, int in_level, u64 *out, long long out_item,
                       int new_level) {
    const long long N = 1ll << c.logN;
    const int item = blockIdx.z;
    const int pl = blockIdx.y;
    const int poly = pl / (new_level + 1), limb = pl % (new_level + 1);
    const u64 *s = in + item * in_item + ((long long)poly * (in_level + 1) + limb) * N;
    u64 *d = out + item * out_item + (long long)pl * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x)
        d[j] = s[j];
}

__global__ void k_decrypt(DevCtx c, const u64 *ct, const u64 *s, u64 *m, int level) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    const ModQ md = c.primes[limb].m;
    const long long off = (long long)limb * N, P = (long long)(level + 1) * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        U128 t = mul_wide(ct[P + off + j], s[off + j]);
        add_to(t, U128{ct[off + j], 0});
        m[off + j] = barrett(t, md);
    }
}

// ---- pt-MAC.  A CTA owns 2 tc consecutive coefficients of one limb for
// 256/tc images (thread = two adjacent coefficients x image, 16-byte loads;
// tc = 32 for 8 or more images, up to 256 for one image, so no thread idles
// on small batches) and computes every output group of the step: the
// rotated inputs it reads stay in L1 across groups, and the CTAs of the image
// tiles of one coefficient tile run back to back so each plaintext tile is
// fetched from HBM once per batch.  Products are summed in 128 bits and
// reduced only when the sum could leave Barrett's range: with b = bitlen(q),
// K products of residues stay below K q^2 < 2^(b+62) for K <= 2^(62-b)
// (16 terms for 58-bit primes).
#ifndef MAC_U
#define MAC_U 2          // single terms whose loads are issued together
#endif
#ifndef MAC_MINB
#define MAC_MINB 3
#endif
__global__ void __launch_bounds__(256, MAC_MINB) k_mac(DevCtx c, MacArgs a, int tc) {
    // each thread owns two adjacent coefficients (16-byte loads)
    const int limb = blockIdx.z;
    const ModQ m = c.primes[a.ext ? ext_prime(limb, a.level, c.L) : limb].m;
    const long long N = 1ll << c.logN;
    const int cl = threadIdx.x % tc, il = threadIdx.x / tc;
    const int img = blockIdx.x * (256 / tc) + il;
    if (img >= a.n_items) return;
    const long long off = (long long)limb * N + (long long)blockIdx.y * 2 * tc + 2 * cl;
    const long long P = (long long)(a.level + 1 + (a.ext ? c.alpha : 0)) * N;
    // products summed before a reduction (one slot kept for the carried residue)
    const int kmax = (m.b >= 61 ? 2 : (1 << min(62 - m.b, 20))) - 1;
    for (int g = 0; g < a.n_groups; g++) {
        const MacGroup G = a.groups[g];
        U128 a00 = {0, 0}, a01 = {0, 0}, a10 = {0, 0}, a11 = {0, 0};   // [poly][coefficient]
        int cnt = 0;
        int t = G.term_begin;
        while (t < G.term_end) {
            const int run = a.terms[t].run;
            bool singles = run <= 1 && t + MAC_U - 1 < G.term_end;
#pragma unroll
            for (int k = 1; k < MAC_U; k++) singles = singles && a.terms[t + min(k, G.term_end - 1 - t)].run <= 1;
            if (singles) {
                // MAC_U single terms: their loads are in flight together
                ulonglong2 p[MAC_U], x0[MAC_U], x1[MAC_U];
#pragma unroll
                for (int k = 0; k < MAC_U; k++) {
                    const MacTerm T = a.terms[t + k];
                    const MacSrc S = a.srcs[T.src];
                    const u64 *sp = S.base + (long long)img * S.item + off;
                    p[k] = __ldg(reinterpret_cast<const ulonglong2 *>(T.pt + off));
                    x0[k] = *reinterpret_cast<const ulonglong2 *>(sp);
                    x1[k] = *reinterpret_cast<const ulonglong2 *>(sp + P);
                }
#pragma unroll
                for (int k = 0; k < MAC_U; k++) {
                    mac(a00, p[k].x, x0[k].x);
                    mac(a01, p[k].y, x0[k].y);
                    mac(a10, p[k].x, x1[k].x);
                    mac(a11, p[k].y, x1[k].y);
                }
                cnt += MAC_U;
                t += MAC_U;
            } else {
                // one term, or a run of terms sharing one plaintext: the
                // run's sources are added mod q (two at a time), then one
                // product
                const MacTerm T = a.terms[t];
                const int len = run < 1 ? 1 : run;
                const u64 *sp = a.srcs[T.src].base + (long long)img * a.srcs[T.src].item + off;
                const ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2 *>(T.pt + off));
                ulonglong2 s0 = *reinterpret_cast<const ulonglong2 *>(sp);
                ulonglong2 s1 = *reinterpret_cast<const ulonglong2 *>(sp + P);
                int r = 1;
                for (; r + 2 <= len; r += 2) {
                    ulonglong2 y0[2], y1[2];
#pragma unroll
                    for (int k = 0; k < 2; k++) {
                        const MacSrc S = a.srcs[a.terms[t + r + k].src];
                        const u64 *q = S.base + (long long)img * S.item + off;
                        y0[k] = *reinterpret_cast<const ulonglong2 *>(q);
                        y1[k] = *reinterpret_cast<const ulonglong2 *>(q + P);
                    }
#pragma unroll
                    for (int k = 0; k < 2; k++) {
                        s0 = make_ulonglong2(add_mod(s0.x, y0[k].x, m.q), add_mod(s0.y, y0[k].y, m.q));
                        s1 = make_ulonglong2(add_mod(s1.x, y1[k].x, m.q), add_mod(s1.y, y1[k].y, m.q));
                    }
                }
                if (r < len) {
                    const MacSrc S = a.srcs[a.terms[t + r].src];
                    const u64 *q = S.base + (long long)img * S.item + off;
                    const ulonglong2 y0 = *reinterpret_cast<const ulonglong2 *>(q);
                    const ulonglong2 y1 = *reinterpret_cast<const ulonglong2 *>(q + P);
                    s0 = make_ulonglong2(add_mod(s0.x, y0.x, m.q), add_mod(s0.y, y0.y, m.q));
                    s1 = make_ulonglong2(add_mod(s1.x, y1.x, m.q), add_mod(s1.y, y1.y, m.q));
                }
                mac(a00, p.x, s0.x);
                mac(a01, p.y, s0.y);
                mac(a10, p.x, s1.x);
                mac(a11, p.y, s1.y);
                cnt += 1;
                t += len;
            }
            // at most MAC_U products before the next check
            if (cnt + MAC_U > kmax) {
                a00 = U128{barrett(a00, m), 0};
                a01 = U128{barrett(a01, m), 0};
                a10 = U128{barrett(a10, m), 0};
                a11 = U128{barrett(a11, m), 0};
                cnt = 0;
            }
        }
        u64 *o = G.out + (long long)img * G.out_item + off;
        const ulonglong2 b = G.bias ? __ldg(reinterpret_cast<const ulonglong2 *>(G.bias + off)) : make_ulonglong2(0, 0);
        ulonglong2 r0 = make_ulonglong2(add_mod(barrett(a00, m), b.x, m.q), add_mod(barrett(a01, m), b.y, m.q));
        ulonglong2 r1 = make_ulonglong2(barrett(a10, m), barrett(a11, m));
        if (G.accumulate) {
            const ulonglong2 o0 = *reinterpret_cast<const ulonglong2 *>(o);
            const ulonglong2 o1 = *reinterpret_cast<const ulonglong2 *>(o + P);
            r0 = make_ulonglong2(add_mod(r0.x, o0.x, m.q), add_mod(r0.y, o0.y, m.q));
            r1 = make_ulonglong2(add_mod(r1.x, o1.x, m.q), add_mod(r1.y, o1.y, m.q));
        }
        *reinterpret_cast<ulonglong2 *>(o) = r0;
        *reinterpret_cast<ulonglong2 *>(o + P) = r1;
    }
}

// ---- on-demand slot encoding (the host encoder's operations, in its order;
// the double-precision intrinsics are never contracted into FMAs)
// row vids[v]'s nonzeros into the bit-reversed FFT input of vector v
// (real parts; the buffer is zeroed first)
__global__ void k_enc_scatter(int n, const int *vids, const long long *begin, const int *slot, const double *val,
                              const unsigned *perm, double *buf) {
    const int v = blockIdx.y;
    const int row = vids[v];
    double *ar = buf + (long long)v * 2 * n;
    for (long long e = begin[row] + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < begin[row + 1];
         e += (long long)gridDim.x * blockDim.x)
        ar[perm[slot[e]]] = val[e];
}

// one radix-2 decimation-in-time stage of length 2^s on every vector
__global__ void k_enc_fft_stage(int n, int s, const double *cr, const double *ci, double *buf) {
    const int v = blockIdx.y;
    double *ar = buf + (long long)v * 2 * n, *ai = ar + n;
    const int half = 1 << (s - 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n / 2; t += gridDim.x * blockDim.x) {
        const int k = t & (half - 1);
        const int j = ((t >> (s - 1)) << s) + k;
        const double wr = cr[k], wi = -ci[k];
        const double br = ar[j + half], bi = ai[j + half];
        const double vr = __dsub_rn(__dmul_rn(br, wr), __dmul_rn(bi, wi));
        const double vi = __dadd_rn(__dmul_rn(br, wi), __dmul_rn(bi, wr));
        const double ur = ar[j], ui = ai[j];
        ar[j] = __dadd_rn(ur, vr);
        ai[j] = __dadd_rn(ui, vi);
        ar[j + half] = __dsub_rn(ur, vr);
        ai[j + half] = __dsub_rn(ui, vi);
    }
}

// twist by exp(-i pi k / N), times scale / n, rounded half away from zero:
// m[k] and m[k + n] overwrite the real and imaginary parts in place
__global__ void k_enc_twist(int n, const double *tc, const double *ts, double f, double *buf) {
    const int v = blockIdx.y;
    double *ar = buf + (long long)v * 2 * n, *ai = ar + n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double c = tc[k], sn = ts[k];
        double r = __dadd_rn(__dmul_rn(ar[k], c), __dmul_rn(ai[k], sn));
        double i = __dsub_rn(__dmul_rn(ai[k], c), __dmul_rn(ar[k], sn));
        r = __dmul_rn(r, f);
        i = __dmul_rn(i, f);
        ar[k] = round(r);
        ai[k] = round(i);
    }
}

// ---- ChaCha20 (RFC 8439 block function)
__device__ __forceinline__ unsigned rotl(unsigned x, int r) { return (x << r) | (x >> (32 - r)); }
#define CQR(a, b, c, d)               \
    a += b; d ^= a; d = rotl(d, 16);  \
    c += d; b ^= c; b = rotl(b, 12);  \
    a += b; d ^= a; d = rotl(d, 8);   \
    c += d; b ^= c; b = rotl(b, 7);

__device__ void chacha_block(uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1, uint32_t ctr,
                             unsigned out[16]) {
    unsigned s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                      (unsigned)seed, (unsigned)(seed >> 32), domain, 0u, 0u, 0u, 0u, 0u,
                      ctr, id0, id1, 0u};
    unsigned x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll
    for (int i = 0; i < 10; i++) {
        CQR(x[0], x[4], x[8], x[12]);
        CQR(x[1], x[5], x[9], x[13]);
        CQR(x[2], x[6], x[10], x[14]);
        CQR(x[3], x[7], x[11], x[15]);
        CQR(x[0], x[5], x[10], x[15]);
        CQR(x[1], x[6], x[11], x[12]);
        CQR(x[2], x[7], x[8], x[13]);
        CQR(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

struct PidxArr {
    unsigned char p[FHE_MAX_LIMBS];
};

// each thread: one block = 4 coefficients of one limb
__global__ void k_sample_uniform(DevCtx c, uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1_base,
                                 uint32_t id1_step, u64 *out, PidxArr pidx) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    const ModQ m = c.primes[pidx.p[limb]].m;
    const u64 r64 = barrett(U128{0, 1}, m);   // 2^64 mod q
    for (long long b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 4; b += (long long)gridDim.x * blockDim.x) {
        unsigned w[16];
        chacha_block(seed, domain, id0, id1_base + (uint32_t)limb * id1_step, (uint32_t)b, w);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const u64 lo = (u64)w[4 * u] | ((u64)w[4 * u + 1] << 32);
            const u64 hi = (u64)w[4 * u + 2] | ((u64)w[4 * u + 3] << 32);
            const u64 h = barrett(U128{hi, 0}, m);
            U128 t = mul_wide(h, r64);
            add_to(t, U128{barrett(U128{lo, 0}, m), 0});
            out[(long long)limb * N + 4 * b + u] = barrett(t, m);
        }
    }
}

// kind 0: ternary (16 coefficients per block), kind 1: CBD eta=21 (8 per block)
__global__ void k_sample_small(DevCtx c, uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1, int kind,
                               long long *out) {
    const long long N = 1ll << c.logN;
    const int per = kind == 0 ? 16 : 8;
    for (long long b = blockIdx.x * blockDim.x + threadIdx.x; b < N / per; b += (long long)gridDim.x * blockDim.x) {
        unsigned w[16];
        chacha_block(seed, domain, id0, id1, (uint32_t)b, w);
        if (kind == 0) {
#pragma unroll
            for (int u = 0; u < 16; u++) out[16 * b + u] = (long long)(((u64)w[u] * 3) >> 32) - 1;
        } else {
#pragma unroll
            for (int u = 0; u < 8; u++)
                out[8 * b + u] = (long long)__popc(w[2 * u] & 0x1FFFFFu) - (long long)__popc(w[2 * u + 1] & 0x1FFFFFu);
        }
    }
}

__global__ void k_signed_to_limbs(DevCtx c, const long long *v, u64 *out, PidxArr pidx) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    const u64 q = c.primes[pidx.p[limb]].m.q;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const long long x = v[j];
        u64 r = x >= 0 ? (u64)x % q : (q - ((u64)(-x) % q)) % q;
        out[(long long)limb * N + j] = r;
    }
}

__global__ void k_mul_limbs(DevCtx c, const u64 *a, const u64 *b, const u64 *add, int negate, u64 *out,
                            PidxArr pidx) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    const ModQ m = c.primes[pidx.p[limb]].m;
    const long long off = (long long)limb * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        u64 p = mulmod(a[off + j], b[off + j], m);
        if (negate) p = p ? m.q - p : 0;
        if (add) p = add_mod(p, add[off + j], m.q);
        out[off + j] = p;
    }
}

__global__ void k_automorphism(DevCtx c, const u64 *in, u64 *out, int galois) {
    const long long N = 1ll << c.logN;
    const long long off = (long long)blockIdx.y * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x)
        out[off + j] = in[off + galois_src((int)j, galois, c.logN)];
}

__global__ void k_axpy_limbs(DevCtx c, const u64 *x, const u64 *cst, u64 *out, PidxArr pidx) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    const ModQ m = c.primes[pidx.p[limb]].m;
    const u64 w = cst[limb];
    const long long off = (long long)limb * N;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x)
        out[off + j] = add_mod(out[off + j], mulmod(x[off + j], w, m), m.q);
}

__device__ u64 pow2_mod(int e, const ModQ &m) {
    u64 r = 1, b = 2 % m.q;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

// exact residue of an integral double: |v| < 2^63 through int64, else as a
// 53-bit integer mantissa times 2^shift
__global__ void k_double_to_limbs(DevCtx c, const double *v, u64 *out, int ext_level) {
    const long long N = 1ll << c.logN;
    const int limb = blockIdx.y;
    // vector blockIdx.z: N doubles in, gridDim.y limbs out
    v += (long long)blockIdx.z * N;
    out += (long long)blockIdx.z * gridDim.y * N;
    const ModQ m = c.primes[ext_level >= 0 ? ext_prime(limb, ext_level, c.L) : limb].m;
    for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const double x = v[j];
        const double ax = fabs(x);
        u64 r;
        if (ax < 9223372036854775808.0) {
            r = (u64)(long long)ax % m.q;
        } else {
            int e;
            const double mant = frexp(ax, &e);
            const u64 mi = (u64)ldexp(mant, 53);
            r = mulmod(mi % m.q, pow2_mod(e - 53, m), m);
        }
        out[(long long)limb * N + j] = (x < 0 && r) ? m.q - r : r;
    }
}

}  // namespace

// ================================================================ launchers

#define DISPATCH_LOGR(logr, KERNEL, GRID, ...)                                      \
    do {                                                                            \
        COUNT_LAUNCH();                                                             \
        switch (logr) {                                                             \
        case 4: KERNEL<4><<<GRID, NT, 0, s>>>(__VA_ARGS__); break;                  \
        case 5: KERNEL<5><<<GRID, NT, 0, s>>>(__VA_ARGS__); break;                  \
        case 6: KERNEL<6><<<GRID, NT, 0, s>>>(__VA_ARGS__); break;                  \
        case 7: KERNEL<7><<<GRID, NT, 0, s>>>(__VA_ARGS__); break;                  \
        case 8: KERNEL<8><<<GRID, NT, 0, s>>>(__VA_ARGS__); break;                  \
        default: return cudaErrorInvalidValue;                                      \
        }                                                                           \
    } while (0)

static inline int tiles_col(const DevCtx &c) { return 1 << (c.logN - 12); }  // CTAs per limb

size_t ks_workspace_words(const DevCtx &c, int level) {
    const int nd = (level + c.alpha) / c.alpha;
    KsLayout L = ks_layout(level, nd, c.alpha, c.logN);
    return (size_t)(L.u + 2ll * (1ll << c.logN));
}

cudaError_t launch_ntt(const DevCtx &c, const NttArgs &a, bool inverse, cudaStream_t s) {
    dim3 g(tiles_col(c), a.n_items * a.n_limbs);
    if (!inverse) {
        DISPATCH_LOGR(c.logR1, k_ntt_fwd_col, g, c, a);
        DISPATCH_LOGR(c.logR2, k_ntt_fwd_row, g, c, a);
    } else {
        DISPATCH_LOGR(c.logR2, k_ntt_inv_row, g, c, a);
        DISPATCH_LOGR(c.logR1, k_ntt_inv_col, g, c, a);
    }
    return cudaGetLastError();
}

static cudaError_t launch_keyswitch_part(const DevCtx &c, const LevelTab &lt, const KsArgs &args, cudaStream_t s,
                                         cudaEvent_t *ev, int phases);

// Grids put items x (rows per item) on grid.y (at most 65535): a batch whose
// ModUp rows (digits x extended limbs per item) exceed that is launched in
// parts of consecutive items (every per-item pointer advanced by its stride).
cudaError_t launch_keyswitch(const DevCtx &c, const LevelTab &lt, const KsArgs &args, cudaStream_t s,
                             cudaEvent_t *ev, int phases) {
    const int nl = args.level + 1;
    const int rows = std::max(std::max(lt.n_digits * lt.ext, 2 * nl), 2 * c.alpha);
    const int per = 65535 / rows;
    if (per < 1) return cudaErrorInvalidValue;
    if (args.n_items <= per) return launch_keyswitch_part(c, lt, args, s, ev, phases);
    for (int i0 = 0; i0 < args.n_items; i0 += per) {
        KsArgs a = args;
        a.n_items = std::min(per, args.n_items - i0);
        if (a.d) a.d = args.d + (long long)i0 * args.d_item;
        if (a.add0) a.add0 = args.add0 + (long long)i0 * args.add_item;
        if (a.add1) a.add1 = args.add1 + (long long)i0 * args.add_item;
        if (a.base) a.base = args.base + (long long)i0 * args.base_item;
        if (a.out) a.out = args.out + (long long)i0 * args.out_item;
        a.ws = args.ws + (long long)i0 * args.ws_item;
        if (a.ip_out) a.ip_out = args.ip_out + (long long)i0 * args.ip_out_item;
        if (a.ip_fold) a.ip_fold = args.ip_fold + (long long)i0 * args.ip_fold_item;
        if (a.md_in) a.md_in = args.md_in + (long long)i0 * args.md_in_item;
        const cudaError_t e = launch_keyswitch_part(c, lt, a, s, i0 == 0 ? ev : nullptr, phases);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_keyswitch_part(const DevCtx &c, const LevelTab &lt, const KsArgs &args, cudaStream_t s,
                                         cudaEvent_t *ev, int phases) {
    KsArgs a = args;
    if (a.ip_galois == 0) a.ip_galois = 1;
    if (a.add_galois == 0) a.add_galois = a.galois;
    const int nl = a.level + 1, ext = lt.ext, nd = lt.n_digits, B = a.n_items;
    if (nd > 64) return cudaErrorInvalidValue;   // the context bounds digits by the primes' sizes
    // the inner product takes two slots per thread: 16-byte aligned operands and
    // N >= 512 (always true of the library's own buffers, whose limbs start at
    // multiples of N)
    if (c.logN < 9 || ((uintptr_t)a.d | (uintptr_t)a.ws | (uintptr_t)a.key) % 16 != 0 || ((a.d_item | a.ws_item) & 1))
        return cudaErrorMisalignedAddress;
    KsLayout ly = ks_layout(a.level, nd, c.alpha, c.logN);
    const int tc = tiles_col(c);
#define KS_EV(i) \
    if (ev) cudaEventRecord(ev[i], s)
    KS_EV(0);
    if (phases & KS_MODUP) DISPATCH_LOGR(c.logR2, k_ks_intt_row, dim3(tc, B * nl), c, a, ly);
    KS_EV(1);
    if (phases & KS_MODUP) DISPATCH_LOGR(c.logR1, k_ks_intt_col, dim3(tc, B * nl), c, lt, a, ly);
    KS_EV(2);
    if (phases & KS_MODUP) DISPATCH_LOGR(c.logR1, k_ks_modup_col, dim3(tc, B * nd * ext), c, lt, a, ly);
    KS_EV(3);
    if (phases & KS_MODUP) DISPATCH_LOGR(c.logR2, k_ks_modup_row, dim3(tc, B * nd * ext), c, lt, a, ly);
    if (phases & KS_IP) {
        COUNT_LAUNCH();
        const dim3 g2((unsigned)((1ll << c.logN) / 512), ext);
        const bool xo = a.ip_out || a.ip_fold;
#define IP_CASE(n)                                                     \
    case n:                                                            \
        if (xo)                                                        \
            k_ks_ip<n, true><<<g2, 256, 0, s>>>(c, lt, a, ly);         \
        else                                                           \
            k_ks_ip<n, false><<<g2, 256, 0, s>>>(c, lt, a, ly);        \
        break;
        switch (nd) {
            IP_CASE(1)
            IP_CASE(2)
            IP_CASE(3)
            IP_CASE(4)
            IP_CASE(5)
            IP_CASE(6)
            IP_CASE(7)
        default: k_ks_ip_n<<<g2, 256, 0, s>>>(c, lt, a, ly);
        }
#undef IP_CASE
    }
    KS_EV(4);
    if (phases & KS_MODDOWN) DISPATCH_LOGR(c.logR2, k_ks_md_intt_row, dim3(tc, B * 2 * c.alpha), c, lt, a, ly);
    KS_EV(5);
    if (phases & KS_MODDOWN) DISPATCH_LOGR(c.logR1, k_ks_md_intt_col, dim3(tc, B * 2 * c.alpha), c, lt, a, ly);
    if (phases & KS_MODDOWN) {
        COUNT_LAUNCH();
        k_ks_md_overflow<<<dim3((unsigned)((1ll << c.logN) / 256), B * 2), 256, 0, s>>>(c, a, ly);
    }
    KS_EV(6);
    if (phases & KS_MODDOWN) DISPATCH_LOGR(c.logR1, k_ks_md_conv_col, dim3(tc, B * 2 * nl), c, lt, a, ly);
    KS_EV(7);
    if (phases & KS_MODDOWN) DISPATCH_LOGR(c.logR2, k_ks_md_row_out, dim3(tc, B * 2 * nl), c, lt, a, ly);
    KS_EV(8);
#undef KS_EV
    return cudaGetLastError();
}

cudaError_t launch_ks_ip_babies(const DevCtx &c, const LevelTab &lt, const KsArgs &a, const IpBabies &bb,
                                cudaStream_t s) {
    const int nd = lt.n_digits;
    if (bb.n < 1 || bb.n > KS_BABIES_MAX || nd < 1 || nd > 7 || c.logN < 9 || !a.ws || !a.d || !a.ip_out_item)
        return cudaErrorInvalidValue;
    if (((uintptr_t)a.d | (uintptr_t)a.ws | (uintptr_t)a.ip_fold) % 16 != 0 ||
        ((a.d_item | a.ws_item | a.ip_fold_item | a.ip_out_item) & 1))
        return cudaErrorMisalignedAddress;
    for (int k = 0; k < bb.n; k++)
        if (!bb.key[k] || !bb.out[k] || ((uintptr_t)bb.key[k] | (uintptr_t)bb.out[k]) % 16 != 0 || !(bb.gal_inv[k] & 1))
            return cudaErrorInvalidValue;
    KsLayout ly = ks_layout(a.level, nd, c.alpha, c.logN);
    const dim3 g((unsigned)((1ll << c.logN) / 512), lt.ext);
    COUNT_LAUNCH();
    switch (nd) {
    case 1: k_ks_ip_babies<1><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    case 2: k_ks_ip_babies<2><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    case 3: k_ks_ip_babies<3><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    case 4: k_ks_ip_babies<4><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    case 5: k_ks_ip_babies<5><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    case 6: k_ks_ip_babies<6><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    default: k_ks_ip_babies<7><<<g, 256, 0, s>>>(c, lt, a, ly, bb); break;
    }
    return cudaGetLastError();
}

static cudaError_t launch_rescale_part(const DevCtx &c, const LevelTab &lt, const RescaleArgs &a, cudaStream_t s);

// Grids put items x polys x limbs on grid.y (at most 65535): larger batches
// are launched in parts of consecutive items.
cudaError_t launch_rescale(const DevCtx &c, const LevelTab &lt, const RescaleArgs &args, cudaStream_t s) {
    if (args.level < 1 || args.n_poly < 1) return cudaErrorInvalidValue;
    const int per = 65535 / (args.n_poly * args.level);
    if (per < 1) return cudaErrorInvalidValue;
    for (int i0 = 0; i0 < args.n_items; i0 += per) {
        RescaleArgs a = args;
        a.n_items = std::min(per, args.n_items - i0);
        a.in = args.in + (long long)i0 * args.in_item;
        a.out = args.out + (long long)i0 * args.out_item;
        a.ws = args.ws + ((long long)i0 * args.n_poly << c.logN);
        const cudaError_t e = launch_rescale_part(c, lt, a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_rescale_part(const DevCtx &c, const LevelTab &lt, const RescaleArgs &a, cudaStream_t s) {
    const int tc = tiles_col(c), B = a.n_items, lv = a.level;
    if (lv < 1) return cudaErrorInvalidValue;
    DISPATCH_LOGR(c.logR2, k_rs_intt_row, dim3(tc, B * a.n_poly), c, a);
    DISPATCH_LOGR(c.logR1, k_rs_intt_col, dim3(tc, B * a.n_poly), c, a);
    DISPATCH_LOGR(c.logR1, k_rs_conv_col, dim3(tc, B * a.n_poly * lv), c, lt, a);
    DISPATCH_LOGR(c.logR2, k_rs_row_out, dim3(tc, B * a.n_poly * lv), c, lt, a);
    return cudaGetLastError();
}

static dim3 ew_grid(const DevCtx &c, int y, int z) {
    int x = (int)((1ll << c.logN) / 256);
    if (x > 64) x = 64;
    return dim3(x, y, z);
}

cudaError_t launch_gather_acc(const DevCtx &c, const u64 *in, long long in_item, u64 *out, long long out_item,
                              int n_items, int level, int galois, int accumulate, cudaStream_t s) {
    COUNT_LAUNCH();
    k_gather_acc<<<ew_grid(c, level + 1, n_items), 256, 0, s>>>(c, in, in_item, out, out_item, level, galois,
                                                                 accumulate);
    return cudaGetLastError();
}

cudaError_t launch_add(const DevCtx &c, const u64 *a, long long a_item, const u64 *b, long long b_item, u64 *out,
                       long long out_item, int n_items, int n_poly, int level, int subtract, cudaStream_t s) {
    COUNT_LAUNCH();
    k_add<<<ew_grid(c, n_poly * (level + 1), n_items), 256, 0, s>>>(c, a, a_item, b, b_item, out, out_item, n_poly,
                                                                     level, subtract);
    return cudaGetLastError();
}

cudaError_t launch_mul_const(const DevCtx &c, const u64 *a, long long a_item, const u64 *cst, u64 *out,
                             long long out_item, int n_items, int n_poly, int level, cudaStream_t s) {
    COUNT_LAUNCH();
    k_mul_const<<<ew_grid(c, n_poly * (level + 1), n_items), 256, 0, s>>>(c, a, a_item, cst, out, out_item, level);
    return cudaGetLastError();
}

cudaError_t launch_add_const(const DevCtx &c, const u64 *a, long long a_item, const u64 *cst, u64 *out,
                             long long out_item, int n_items, int level, cudaStream_t s) {
    COUNT_LAUNCH();
    k_add_const<<<ew_grid(c, 2 * (level + 1), n_items), 256, 0, s>>>(c, a, a_item, cst, out, out_item, level);
    return cudaGetLastError();
}

cudaError_t launch_square_act(const DevCtx &c, const u64 *in, long long in_item, const u64 *c1, const u64 *c0,
                              u64 *out, long long out_item, int n_items, int level, cudaStream_t s, const u64 *c1v,
                              const u64 *c0v, int n_ct) {
    if ((c1v == nullptr) != (c0v == nullptr) || n_ct < 1) return cudaErrorInvalidValue;
    COUNT_LAUNCH();
    k_square_act<<<ew_grid(c, level + 1, n_items), 256, 0, s>>>(c, in, in_item, c1, c0, out, out_item, level, c1v,
                                                                 c0v, n_ct);
    return cudaGetLastError();
}

cudaError_t launch_drop(const DevCtx &c, const u64 *in, long long in_item, int in_level, u64 *out,
                        long long out_item, int new_level, int n_items, int n_poly, cudaStream_t s) {
    COUNT_LAUNCH();
    k_drop<<<ew_grid(c, n_poly * (new_level + 1), n_items), 256, 0, s>>>(c, in, in_item, in_level, out, out_item,
                                                                          new_level);
    return cudaGetLastError();
}

cudaError_t launch_decrypt(const DevCtx &c, const u64 *ct, const u64 *s_ntt, u64 *m, int level, cudaStream_t s) {
    COUNT_LAUNCH();
    k_decrypt<<<ew_grid(c, level + 1, 1), 256, 0, s>>>(c, ct, s_ntt, m, level);
    return cudaGetLastError();
}

cudaError_t launch_mac(const DevCtx &c, const MacArgs &a, cudaStream_t s) {
    if (a.n_groups == 0) return cudaSuccess;
    // images per CTA: as asked, else the batch rounded up to a power of two,
    // at most 8
    int ib = a.images_per_cta;
    if (ib == 0)
        for (ib = 1; ib < 8 && ib < a.n_items;) ib *= 2;
    if (ib != 1 && ib != 2 && ib != 4 && ib != 8) return cudaErrorInvalidValue;
    const int tc = 256 / ib;   // threads per image, two coefficients each
    if ((1ll << c.logN) % (2 * tc)) return cudaErrorInvalidValue;
    dim3 g((a.n_items + ib - 1) / ib, (unsigned)((1ll << c.logN) / (2 * tc)), a.level + 1 + (a.ext ? c.alpha : 0));
    COUNT_LAUNCH();
    k_mac<<<g, 256, 0, s>>>(c, a, tc);
    return cudaGetLastError();
}

static PidxArr to_pidx(const unsigned char *p, int n) {
    PidxArr r;
    for (int i = 0; i < FHE_MAX_LIMBS; i++) r.p[i] = i < n ? p[i] : 0;
    return r;
}

cudaError_t launch_sample_uniform(const DevCtx &c, uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1_base,
                                  uint32_t id1_step, u64 *out, int n_limbs, const unsigned char *pidx,
                                  cudaStream_t s) {
    COUNT_LAUNCH();
    k_sample_uniform<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, seed, domain, id0, id1_base, id1_step, out,
                                                             to_pidx(pidx, n_limbs));
    return cudaGetLastError();
}

cudaError_t launch_sample_small(const DevCtx &c, uint64_t seed, uint32_t domain, uint32_t id0, uint32_t id1, int kind,
                                long long *out, cudaStream_t s) {
    COUNT_LAUNCH();
    k_sample_small<<<ew_grid(c, 1, 1), 256, 0, s>>>(c, seed, domain, id0, id1, kind, out);
    return cudaGetLastError();
}

cudaError_t launch_signed_to_limbs(const DevCtx &c, const long long *v, u64 *out, int n_limbs,
                                   const unsigned char *pidx, cudaStream_t s) {
    COUNT_LAUNCH();
    k_signed_to_limbs<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, v, out, to_pidx(pidx, n_limbs));
    return cudaGetLastError();
}

cudaError_t launch_mul_limbs(const DevCtx &c, const u64 *a, const u64 *b, const u64 *add, int negate, u64 *out,
                             int n_limbs, const unsigned char *pidx, cudaStream_t s) {
    COUNT_LAUNCH();
    k_mul_limbs<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, a, b, add, negate, out, to_pidx(pidx, n_limbs));
    return cudaGetLastError();
}

cudaError_t launch_axpy_limbs(const DevCtx &c, const u64 *x, const u64 *cst, u64 *out, int n_limbs,
                              const unsigned char *pidx, cudaStream_t s) {
    COUNT_LAUNCH();
    k_axpy_limbs<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, x, cst, out, to_pidx(pidx, n_limbs));
    return cudaGetLastError();
}

cudaError_t launch_double_to_limbs(const DevCtx &c, const double *v, u64 *out, int n_limbs, cudaStream_t s,
                                   int ext_level) {
    COUNT_LAUNCH();
    k_double_to_limbs<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, v, out, ext_level);
    return cudaGetLastError();
}

cudaError_t launch_encode_sparse(const DevCtx &c, const EncTab &e, int V, const int *vids, const long long *begin,
                                 const int *slot, const double *val, double scale, int level, double *buf, u64 *pt,
                                 cudaStream_t s, bool ext) {
    if (V <= 0) return cudaSuccess;
    const int n_limbs = level + 1 + (ext ? c.alpha : 0);
    if (V > 65535 || n_limbs > FHE_MAX_LIMBS) return cudaErrorInvalidValue;
    const int n = 1 << (c.logN - 1);
    cudaError_t r = cudaMemsetAsync(buf, 0, (size_t)V * 2 * n * sizeof(double), s);
    if (r != cudaSuccess) return r;
    COUNT_LAUNCH();
    k_enc_scatter<<<dim3(4, V), 256, 0, s>>>(n, vids, begin, slot, val, e.perm, buf);
    const int bx = std::min(n / 2 / 256 > 0 ? n / 2 / 256 : 1, 64);
    for (int st = 1; (1 << st) <= n; st++) {
        COUNT_LAUNCH();
        k_enc_fft_stage<<<dim3(bx, V), 256, 0, s>>>(n, st, e.fft_re + e.off[st], e.fft_im + e.off[st], buf);
    }
    COUNT_LAUNCH();
    k_enc_twist<<<dim3(bx, V), 256, 0, s>>>(n, e.tw_c, e.tw_s, scale / (double)n, buf);
    COUNT_LAUNCH();
    k_double_to_limbs<<<dim3(std::min((int)((1ll << c.logN) / 256), 64), n_limbs, V), 256, 0, s>>>(
        c, buf, pt, ext ? level : -1);
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = pt;
    a.dst = pt;
    a.src_item = a.dst_item = (long long)n_limbs << c.logN;
    a.n_items = V;
    a.n_limbs = n_limbs;
    for (int l = 0; l < n_limbs; l++) a.pidx[l] = (unsigned char)ext_prime(l, ext ? level : c.L, c.L);
    return launch_ntt(c, a, false, s);
}

cudaError_t launch_automorphism(const DevCtx &c, const u64 *in, u64 *out, int n_limbs, int galois, cudaStream_t s) {
    COUNT_LAUNCH();
    k_automorphism<<<ew_grid(c, n_limbs, 1), 256, 0, s>>>(c, in, out, galois);
    return cudaGetLastError();
}
