// Rescale for callers that must not allocate device memory.
//
// The regular rescale takes its scratch (the inverse NTT of the top limb of
// each polynomial) from a workspace the library grows with cudaMalloc.  Some
// callers cannot let a library do that: an application that hands the GPU's
// memory to its own pool or to a framework up front and forbids any further
// driver allocation, a latency-critical loop that must not hit cudaMalloc's
// implicit device synchronisation, or a process running under a fixed memory
// budget.  fhe_rescale_noalloc serves them: the caller passes device input
// and output buffers, and the scratch is the file-scope device array below,
// of a fixed size.  Every GPU that loads the library keeps that array until
// the process exits.
#include <mutex>

#include "host.h"

// room for two polynomials of N = 2^16 (1 MiB)
#define FHE_NOALLOC_SCRATCH_WORDS (2ull << 16)

static __device__ __align__(256) u64 g_noalloc_scratch[FHE_NOALLOC_SCRATCH_WORDS];

// Device address of the array, one per device.  In host code the array's name
// is only a stand-in for the symbol, never an address a kernel may use.
#define FHE_NOALLOC_MAX_DEVICES 64
static std::mutex g_noalloc_mu;
static u64 *g_noalloc_addr[FHE_NOALLOC_MAX_DEVICES] = {nullptr};

static int noalloc_scratch(int dev, u64 **out) {
    if (dev < 0 || dev >= FHE_NOALLOC_MAX_DEVICES) return fhe_fail(FHE_E_INVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        // the context's device is current here
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fhe_fail(FHE_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = (u64 *)p;
    }
    *out = g_noalloc_addr[dev];
    return FHE_OK;
}

extern "C" int fhe_rescale_noalloc(fhe_ctx *c, const uint64_t *in, uint64_t *out, int n_poly, int level,
                                   void *stream) {
    if (!c || !in || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    if (level < 1 || level > c->L) return fhe_fail(FHE_E_LEVEL, "level must be in [1, L]");
    if (n_poly < 1 || n_poly > 3) return fhe_fail(FHE_E_INVAL, "n_poly must be 1..3");
    if ((unsigned long long)n_poly * (unsigned long long)c->N > FHE_NOALLOC_SCRATCH_WORDS)
        return fhe_fail(FHE_E_INVAL, "n_poly * N exceeds the fixed scratch of " +
                                         std::to_string(FHE_NOALLOC_SCRATCH_WORDS) + " words");
    const u64 *ib = (const u64 *)in, *ie = ib + (size_t)n_poly * (level + 1) * c->N;
    const u64 *ob = (const u64 *)out, *oe = ob + (size_t)n_poly * level * c->N;
    if (ib < oe && ob < ie) return fhe_fail(FHE_E_INVAL, "input and output buffers overlap");
    FHE_CU(cudaSetDevice(c->dev));
    u64 *scratch;
    FHE_TRY(noalloc_scratch(c->dev, &scratch));
    RescaleArgs a;
    a.in = (const u64 *)in;
    a.in_item = 0;
    a.out = (u64 *)out;
    a.out_item = 0;
    a.n_items = 1;
    a.n_poly = n_poly;
    a.level = level;
    a.ws = scratch;
    FHE_CU(launch_rescale(c->dc, c->lt[level], a, (cudaStream_t)stream));
    return FHE_OK;
}
