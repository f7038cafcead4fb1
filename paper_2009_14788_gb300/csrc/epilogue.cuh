// Device side of the projector output epilogue (struct Epilogue in radon_internal.h).
#pragma once

#include "dtype.cuh"
#include "radon_internal.h"

namespace radon {

// op_scale * s * p + add_scale * add[idx], in FP32; the caller rounds once to the storage type.
template <typename T>
__device__ __forceinline__ float epilogue_value(const Epilogue& ep, float p, long long idx) {
    float v = p * ep.op_scale;
    if (ep.op_scale_dev != nullptr) v *= *ep.op_scale_dev;
    if (ep.add != nullptr) v = fmaf(ep.add_scale, to_f32(static_cast<const T*>(ep.add)[idx]), v);
    return v;
}

// The same with the storage type chosen at run time (kernels not templated on it).
__device__ __forceinline__ void epilogue_store_rt(const Epilogue& ep, int dtype, void* out, float p, long long idx) {
    if (dtype == RADON_F16) {
        static_cast<__half*>(out)[idx] = __float2half_rn(epilogue_value<__half>(ep, p, idx));
    } else if (dtype == RADON_BF16) {
        static_cast<__nv_bfloat16*>(out)[idx] = __float2bfloat16_rn(epilogue_value<__nv_bfloat16>(ep, p, idx));
    } else {
        static_cast<float*>(out)[idx] = epilogue_value<float>(ep, p, idx);
    }
}

}  // namespace radon
