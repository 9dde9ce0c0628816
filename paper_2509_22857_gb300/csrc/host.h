// Host-side internals shared by the library's translation units.
#pragma once
#include <cstdint>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/fhecnn.h"
#include "kernels.h"

typedef unsigned __int128 u128;

int fhe_fail(int code, const std::string &msg);

#define FHE_CU(call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// a stream-ordered allocation: refusal is FHE_E_OOM, as for dev_alloc
#define FHE_ALLOC_ASYNC(ptr, bytes, stream)                                                        \
    do {                                                                                           \
        cudaError_t e_ = cudaMallocAsync((void **)(ptr), (bytes), (stream));                       \
        if (e_ == cudaErrorMemoryAllocation) {                                                     \
            cudaGetLastError();                                                                    \
            return fhe_fail(FHE_E_OOM, "cudaMallocAsync(" + std::to_string((size_t)(bytes)) + "): out of memory"); \
        }                                                                                          \
        if (e_ != cudaSuccess) return fhe_fail(FHE_E_CUDA, std::string("cudaMallocAsync: ") + cudaGetErrorString(e_)); \
    } while (0)

#define FHE_TRY(call)              \
    do {                           \
        int r_ = (call);           \
        if (r_ != FHE_OK) return r_; \
    } while (0)

// ---- host modular arithmetic
inline u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_powmod(u64 a, u64 e, u64 q);
inline u64 h_invmod(u64 a, u64 q) { return h_powmod(a % q, q - 2, q); }
inline u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
bool h_is_prime(u64 n);
std::vector<u64> h_gen_primes(int bits, int count, u64 two_n, const std::vector<u64> &taken);
u64 h_root_2n(u64 q, u64 two_n);

// ---- slot encoder / decoder (host FFT)
struct Encoder {
    int logN = 0;
    size_t N = 0, n = 0;
    std::vector<double> fft_re, fft_im;   // per stage length, concatenated: len/2 entries each
    std::vector<size_t> fft_off;          // offset of stage with length 2^s
    std::vector<double> tw_c, tw_s;       // cos, sin(pi k / N)
    std::vector<uint32_t> slot_pos;       // t_j = (5^j mod 2N - 1) / 4
    std::vector<uint32_t> brv;            // bit reversal over log2(n) bits
    void init(int logN);
    // integral doubles m[N] = round(scale * sigma^-1(z))
    void encode(const double *re, const double *im, size_t nz, double scale, double *m) const;
    // slots from real coefficients (centred values) divided by scale
    void decode(const double *m, double scale, double *re, double *im, size_t nz) const;
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct fhe_ctx {
    fhe_params prm;
    int logN = 0, L = 0, alpha = 0, n_primes = 0;
    long long N = 0;
    double scale = 0;
    std::vector<u64> primes;          // q_0..q_L, p_0..
    DevCtx dc;
    std::vector<LevelTab> lt;         // per level
    std::vector<void *> owned;        // device allocations of the context
    Encoder enc;
    // growable workspaces
    u64 *ks_ws = nullptr;
    size_t ks_ws_words = 0;
    u64 *rs_ws = nullptr;
    size_t rs_ws_words = 0;
    int dev = 0;
    int lin_chunk_srcs = 160;         // MAC sources per chunk of a linear step
    size_t on_demand_bytes = 4ull << 30;   // scratch of plaintexts encoded on demand (per linear step)
    int ks_item_cap = 0;              // whole key switches in launches of at most this many items (0: any)
    int mac_images = 0;               // images per plaintext-MAC CTA (0: the batch rounded up to 2^k, <= 8)
    std::atomic<int> fail_alloc_after{-1};   // injected failure: allocations left before one is refused
    EncTab enc_dev;                   // device copy of the encoder's tables (on first use)
    bool enc_dev_ready = false;
};

struct fhe_ct {
    fhe_ctx *ctx;
    u64 *d;
    int level, n_poly;
    double scale;
};

struct fhe_pt {
    fhe_ctx *ctx;
    u64 *d;       // NTT-domain limbs 0..level
    int level;
    double scale;
};

struct fhe_sk {
    fhe_ctx *ctx;
    u64 *s_ntt;   // [L+1+alpha][N]
};

struct fhe_evk {
    fhe_ctx *ctx;
    int digits;                   // digits at the top level
    u64 *relin = nullptr;         // [digits][2][L+1+alpha][N]
    std::map<int, u64 *> galois;  // Galois element -> key
};

// hand the current device's stream-ordered pool memory that is not in use
// back to the device (after a device synchronisation)
cudaError_t pool_trim();
int dev_alloc(fhe_ctx *ctx, void **p, size_t bytes);
void dev_free(void *p);
int ws_reserve(fhe_ctx *ctx, u64 **ws, size_t *have, size_t words);
int galois_of_step(const fhe_ctx *ctx, int step);
size_t key_words(const fhe_ctx *ctx);

// integral double -> residue mod q (exact)
u64 h_double_mod(double v, u64 q);

// core operations on raw device buffers (batched over items)
// ws: caller-sized workspace, or nullptr for the context's growable one
// phases: KS_MODUP | KS_IP | KS_MODDOWN (the workspace carries state between them)
int op_keyswitch(fhe_ctx *ctx, KsArgs a, cudaStream_t s, u64 *ws = nullptr, int phases = KS_ALL);
// inner products of several baby-step rotations of the ModUp just made in
// ws (the context's workspace when null), each kept in Q_l u P
int op_ks_ip_babies(fhe_ctx *ctx, KsArgs a, const IpBabies &bb, cudaStream_t s, u64 *ws = nullptr);
int op_rescale(fhe_ctx *ctx, const u64 *in, long long in_item, u64 *out, long long out_item, int n_items,
               int n_poly, int level, cudaStream_t s, u64 *ws = nullptr);
int op_ntt(fhe_ctx *ctx, const u64 *src, u64 *dst, long long item, int n_items, int n_limbs,
           const unsigned char *pidx, bool inverse, cudaStream_t s);
// the encoder's tables on the device, uploaded on the first call
int enc_tables(fhe_ctx *ctx, const EncTab **out);
// encode integral doubles into NTT-domain limbs 0..level (device)
// ext: the level+1+alpha limbs of Q_level u P (else limbs 0..level)
int op_encode_to(fhe_ctx *ctx, const double *m_host, int level, u64 *dst, cudaStream_t s, bool ext = false);
