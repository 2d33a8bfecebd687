// tt_gram_noalloc: the left Gram G = A^T A without any device allocation.
//
// Who needs this: callers that must not allocate device memory themselves or
// through this library -- for example a host application whose own allocator
// owns all of the device's memory and forbids allocations behind its back, or
// a latency-critical loop where the implicit synchronisation of cudaMalloc and
// cudaFree is not acceptable.  tt_gram obtains its split-K scratch from the
// stream-ordered allocator; this variant instead uses one fixed array in device
// global memory that is part of the library image.
//
// Scratch: g_gram_scratch below, 2^20 doubles (8 MiB), allocated by the CUDA
// module loader on every GPU that loads the library and held until the process
// exits.  The split-K factor is chosen so that the partial Gram matrices fit in
// it, which limits n (the number of columns) to 1024.
//
// The host cannot use the symbol name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; that first call should therefore come before any
// stream capture starts.  All calls share the one array: calls that overlap on
// the GPU (different streams, or different host threads on one device) race on
// it and must be serialised by the caller.  Nothing in the array needs clearing
// between calls: every entry a call reads is written earlier in the same call.
#include <mutex>

#include "internal.h"

namespace ttsn {
namespace {

constexpr size_t GRAM_SCRATCH_DOUBLES = size_t(1) << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_gram_scratch[GRAM_SCRATCH_DOUBLES];

std::mutex g_lock;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};

tt_status scratch_address(double** out) {
    int dev = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("tt_gram_noalloc: device index out of range");
        return TT_ERR_ARG;
    }
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error(std::string("tt_gram_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return TT_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return TT_OK;
}

}  // namespace
}  // namespace ttsn

using namespace ttsn;

extern "C" tt_status tt_gram_noalloc(int m, int n, const double* A, int lda, double* G, int ldg,
                                     void* stream) {
    set_error("");
    if (m < 0 || n < 0) {
        set_error("tt_gram_noalloc: negative size");
        return TT_ERR_ARG;
    }
    if (n == 0) return TT_OK;
    if (!A || !G) {
        set_error("tt_gram_noalloc: null pointer");
        return TT_ERR_ARG;
    }
    if (lda < n || ldg < n) {
        set_error("tt_gram_noalloc: leading dimension smaller than n");
        return TT_ERR_ARG;
    }
    if ((size_t)n * (size_t)n > GRAM_SCRATCH_DOUBLES) {
        set_error("tt_gram_noalloc: n = " + std::to_string(n) +
                  " exceeds the fixed scratch limit (n <= 1024); use tt_gram");
        return TT_ERR_TOO_LARGE;
    }
    double* scratch = nullptr;
    TT_TRY(scratch_address(&scratch));
    return gram_fixed_scratch((cudaStream_t)stream, m, n, A, lda, G, ldg, scratch,
                              GRAM_SCRATCH_DOUBLES);
}
