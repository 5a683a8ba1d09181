// Internal helpers of the nas library: error handling, RAII device buffers,
// timing.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/nas.h"

namespace nas {

// Internal failures travel as exceptions and are turned into NAS_E_* codes at
// the C ABI boundary (capi.cpp).
struct Error : public std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error(code, msg); }

#define NAS_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            ::nas::fail(NAS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// kernels launched by this library from the calling host thread (counted at
// every launch site; per thread, so concurrent contexts count separately)
extern thread_local long long g_launch_count;

#define NAS_CHECK_LAUNCH()                 \
    do {                                   \
        ++::nas::g_launch_count;           \
        NAS_CUDA(cudaGetLastError());      \
    } while (0)

// Device buffer owned by the library.
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            fail(NAS_E_OOM, std::string("cudaMalloc(") + std::to_string(count * sizeof(T)) +
                                " bytes): " + cudaGetErrorString(e));
        }
        n = count;
    }
    void ensure(size_t count) { if (n < count) alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const T* h, size_t count, cudaStream_t s) {
        ensure(count);
        if (count) NAS_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void upload(const std::vector<T>& h, cudaStream_t s) { upload(h.data(), h.size(), s); }
    void download(T* h, size_t count, cudaStream_t s) const {
        if (count) NAS_CUDA(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
    void zero(cudaStream_t s) {
        if (n) NAS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
};

inline double wall_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647LL;
    return static_cast<int>(g);
}

}  // namespace nas
