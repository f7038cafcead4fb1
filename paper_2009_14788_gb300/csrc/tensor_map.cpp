// Host-side TMA descriptor encoding.  cuTensorMapEncodeTiled is a driver entry point; it is
// fetched through the runtime so the library needs no link-time dependency on libcuda.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "tensor_map.h"

namespace radon {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn g_encode = nullptr;
std::once_flag g_once;

void resolve() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess) {
        g_encode = (EncodeTiledFn)fn;
    }
}

}  // namespace

int encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* base, const uint64_t* dims,
                 const uint64_t* strides_bytes, const uint32_t* box, CUtensorMapL2promotion l2) {
    std::call_once(g_once, resolve);
    if (g_encode == nullptr) return -1;
    cuuint64_t gd[5], gs[5] = {0, 0, 0, 0, 0};
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i > 0) gs[i - 1] = strides_bytes[i - 1];
    }
    CUresult r = g_encode(map, dt, (cuuint32_t)rank, base, gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, l2, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (int)r;
}

CUtensorMapDataType tma_dtype(radon_dtype dt) {
    switch (dt) {
        case RADON_F16: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        case RADON_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    }
}

}  // namespace radon
