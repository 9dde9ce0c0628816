// Host check of the library's modular arithmetic (compiled with g++ by
// tests/test_modarith_host.py): Barrett reduction of sums of up to eight
// products and Shoup multiplication against 128-bit '%', for primes of
// 20..58 bits (the library's limits for explicit chains); and the key inner
// product's sums of one product per digit at the context's digit cap
// min(2^(62 - b), 64), worst case and random.  Prints "ok" or the first
// failure.
#include <cstdio>
#include <random>
#include "../paper_2509_22857_gb300/csrc/modarith.cuh"

typedef unsigned __int128 u128;

static bool is_prime(u64 n) {
    if (n < 2) return false;
    for (u64 p = 2; p < 1000 && p * p <= n; p++)
        if (n % p == 0) return n == p;
    // Miller-Rabin with the first twelve prime bases
    u64 d = n - 1; int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    auto pw = [&](u64 a, u64 e) { u64 x = 1; a %= n; while (e) { if (e & 1) x = (u128)x * a % n; a = (u128)a * a % n; e >>= 1; } return x; };
    for (u64 a : {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37}) {
        u64 x = pw(a, d);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r && comp; i++) { x = (u128)x * x % n; if (x == n - 1) comp = false; }
        if (comp) return false;
    }
    return true;
}

int main() {
    std::mt19937_64 g(12345);
    for (int bits = 20; bits <= 58; bits++) {
        for (int rep = 0; rep < 3; rep++) {
            u64 q = ((1ull << bits) - 1) - (g() % (1ull << (bits - 2)));
            q |= 1;
            while (!is_prime(q)) q -= 2;
            ModQ m;
            m.q = q;
            m.b = 64 - __builtin_clzll(q);
            m.mu = (u64)(((u128)1 << (m.b + 62)) / q);
            for (int it = 0; it < 20000; it++) {
                int terms = 1 + (int)(g() % 8);
                U128 acc = {0, 0};
                u128 ref = 0;
                for (int t = 0; t < terms; t++) {
                    u64 a = g() % q, b = g() % q;
                    mac(acc, a, b);
                    ref += (u128)a * b;
                }
                u64 r = barrett(acc, m);
                if (r != (u64)(ref % q)) { printf("barrett fail q=%llu terms=%d\n", q, terms); return 1; }
                u64 w = g() % q, wp = (u64)(((u128)w << 64) / q), a = g();
                u64 s = mul_shoup(a % (4 * q > q ? 4 * q : q), w, wp, q);
                if (s != (u64)((u128)(a % (4 * q > q ? 4 * q : q)) * w % q)) { printf("shoup fail\n"); return 1; }
                // sums of up to eight products of a residue of a 58-bit prime
                // and a residue of q (basis conversions), and a 64-bit word
                U128 acc2 = {0, 0};
                u128 ref2 = 0;
                for (int t = 0; t < terms; t++) {
                    u64 a = g() >> 6, b = g() % q;
                    mac(acc2, a, b);
                    ref2 += (u128)a * b;
                }
                if (barrett(acc2, m) != (u64)(ref2 % q)) { printf("wide-sum fail q=%llu\n", q); return 1; }
                u64 word = g();
                if (barrett(U128{word, 0}, m) != word % q) { printf("word reduction fail\n"); return 1; }
            }
            // key inner product: one product of two residues per digit, as many
            // digits as the context admits for this prime size
            const int dmax = bits >= 56 ? (1 << (62 - bits)) : 64;
            for (int it = 0; it < 500; it++) {
                U128 acc = {0, 0};
                u128 ref = 0;
                for (int t = 0; t < dmax; t++) {
                    const u64 a = it == 0 ? q - 1 : g() % q, b = it == 0 ? q - 1 : g() % q;
                    mac(acc, a, b);
                    ref += (u128)a * b;
                }
                if (barrett(acc, m) != (u64)(ref % q)) { printf("digit-sum fail q=%llu digits=%d\n", q, dmax); return 1; }
            }
        }
    }
    printf("ok\n");
    return 0;
}
