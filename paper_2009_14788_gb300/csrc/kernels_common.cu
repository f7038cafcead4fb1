// The library's device error word.  Kernels that bound their waits or check their own
// indices record the first failure here (atomicCAS from 0); the host reads and clears it
// through radon_get_device_error.
#include <mutex>

#include "device_error.cuh"
#include "radon_internal.h"

namespace radon {

__device__ int g_device_error = 0;

cudaError_t read_and_clear_device_error(int* out) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_error, sizeof(int));
    if (e != cudaSuccess) return e;
    if (v != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int));
        if (e != cudaSuccess) return e;
    }
    *out = v;
    return cudaSuccess;
}

cudaError_t device_error_address(int** out) {
    // The symbol's device address, looked up with the calling device current (each device that
    // loads the library has its own copy of the word).
    return cudaGetSymbolAddress((void**)out, g_device_error);
}

int* device_error_word() {
    // one copy of the word per device; looked up once per device with that device current
    static std::mutex mu;
    static int* cached[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == nullptr) {
        int* p = nullptr;
        if (device_error_address(&p) != cudaSuccess) return nullptr;
        cached[dev] = p;
    }
    return cached[dev];
}

}  // namespace radon
