// Weighted column dot products without any device allocation.
//
// nas_coldot_f64 takes its scratch (the per-block partial sums) from the
// stream-ordered allocator on every call.  Some callers cannot allocate at
// the point where they need the reduction: an application that has already
// handed all device memory to its own pool allocator (so a library
// allocation would fail or fragment that pool), a latency-critical loop in
// which an allocator call may block or synchronise, or code that must not
// gain a new out-of-memory failure point in the middle of a long run.  This
// entry point serves them: its scratch is a fixed array in device global
// memory that is part of the library image, so a call allocates nothing.
//
// Costs and rules of that array:
//  * it is file-scope (static __device__), kNoAllocMaxCols * 1216 doubles
//    (608 KiB), and every GPU that loads the library holds it until the
//    process exits;
//  * host code cannot use the array's name as a device address (the host
//    symbol is only a stand-in); the device address is looked up once per
//    device with cudaGetSymbolAddress, the first time this entry point runs
//    on that device, with that device current.  That first call performs
//    this set-up and should therefore come before any stream capture.  The
//    address belongs to the device's primary context: after cudaDeviceReset
//    (or anything else that destroys that context) the cached address is
//    stale, so a process that resets a device must not call this entry
//    point on it again;
//  * all calls share the one array: calls that overlap on the GPU (on
//    different streams, or from different host threads) race and may return
//    wrong sums.  Serialise them, e.g. on one stream.  Each call writes every
//    partial sum it later reads, so nothing needs clearing between calls.
#include <mutex>

#include "kernels.h"

namespace {

constexpr int kNoAllocMaxCols = 64;
constexpr int kNoAllocPartials = 1216 * kNoAllocMaxCols;  // partial sums of one call

static __device__ __align__(256) double g_coldot_scratch[kNoAllocPartials];

std::mutex g_scratch_mu;
double* g_scratch_ptr[256] = {};  // device address of g_coldot_scratch, per device

}  // namespace

extern "C" int nas_coldot_f64_noalloc(int64_t n, int N, const double* X, const double* Y, const double* w,
                                      double* out, void* stream) {
    if (n < 0 || !X || !Y || !out) return NAS_E_INVALID_ARG;
    if (N < 1 || N > kNoAllocMaxCols) return NAS_E_INVALID_ARG;
    if (nas::reduce_partial_size(N) > kNoAllocPartials) return NAS_E_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NAS_E_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_coldot_scratch) != cudaSuccess || !p) return NAS_E_CUDA;
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    try {
        const double* Xs[1] = {X};
        const double* Ys[1] = {Y};
        nas::launch_coldots(n, N, 1, Xs, Ys, w, scratch, out, static_cast<cudaStream_t>(stream));
    } catch (const nas::Error& e) {
        return e.code;
    }
    return NAS_OK;
}
