// Device-side error reporting shared by the kernel translation units (relocatable device code
// is not used: each kernel file receives the address of the error word as an argument).
#pragma once

namespace radon {

// Record `code` (a radon_status) if no earlier error is pending.
__device__ __forceinline__ void record_device_error(int* word, int code) {
    atomicCAS(word, 0, code);
}

}  // namespace radon
