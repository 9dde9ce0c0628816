// 64-bit modular arithmetic for primes q < 2^58 on the integer pipes.
//
// * Shoup multiplication by a precomputed constant w (w' = floor(w 2^64 / q)):
//   one high and two low 64-bit products, result in [0, 2q).
// * Barrett reduction of a 128-bit accumulator x < 2^(b+62), b = bitlen(q):
//   with A = b-2 and mu = floor(2^(b+62) / q) (< 2^63), the estimate
//   floor(floor(x / 2^A) * mu / 2^64) -- one high product -- is at most 2
//   below floor(x / q): its error is below x/2^(b+62) + 2^A/q + 1 < 2.5.
//   So x - estimate*q lies in [0, 3q) and two conditional subtractions
//   finish.  floor(x / 2^A) < 2^64 holds because x < 2^(b+62).  For b <= 58
//   this admits any 64-bit word, eight products of residues of q, or sums of
//   up to eight products of a 58-bit residue and a residue of q.
#pragma once
#include <cstdint>

typedef unsigned long long u64;

#ifdef __CUDACC__
#define FHE_HD __host__ __device__ __forceinline__
#else
#define FHE_HD inline
#endif

FHE_HD u64 umulhi64(u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}

struct ModQ {
    u64 q;
    u64 mu;      // floor(2^(b+62) / q)
    int b;       // bit length of q
    int pad_;
};

struct U128 {
    u64 lo, hi;
};

FHE_HD U128 mul_wide(u64 a, u64 b) {
    U128 r;
    r.lo = a * b;
    r.hi = umulhi64(a, b);
    return r;
}

FHE_HD void add_to(U128 &acc, U128 v) {
    u64 lo = acc.lo + v.lo;
    acc.hi += v.hi + (lo < acc.lo ? 1ull : 0ull);
    acc.lo = lo;
}

FHE_HD void mac(U128 &acc, u64 a, u64 b) { add_to(acc, mul_wide(a, b)); }

FHE_HD u64 barrett(U128 x, const ModQ &m) {
    const int A = m.b - 2;
    const u64 x1 = (x.lo >> A) | (x.hi << (64 - A));
    const u64 est = umulhi64(x1, m.mu);
    u64 r = x.lo - est * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}

FHE_HD u64 mulmod(u64 a, u64 b, const ModQ &m) { return barrett(mul_wide(a, b), m); }

FHE_HD u64 mul_shoup_lazy(u64 a, u64 w, u64 wp, u64 q) {
    u64 qh = umulhi64(a, wp);
    return a * w - qh * q;  // in [0, 2q)
}

FHE_HD u64 mul_shoup(u64 a, u64 w, u64 wp, u64 q) {
    u64 r = mul_shoup_lazy(a, w, wp, q);
    return r >= q ? r - q : r;
}

FHE_HD u64 add_mod(u64 a, u64 b, u64 q) {
    u64 r = a + b;
    return r >= q ? r - q : r;
}

FHE_HD u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

FHE_HD u64 reduce_4q(u64 a, u64 q) {
    if (a >= 2 * q) a -= 2 * q;
    if (a >= q) a -= q;
    return a;
}
