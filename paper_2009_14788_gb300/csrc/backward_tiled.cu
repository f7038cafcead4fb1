// Host launcher and instantiations of the tiled gather adjoint (backward_tiled.cuh).
#include <cmath>
#include <cstdlib>

#include "backward_tiled.cuh"
#include "tensor_map.h"

namespace radon {

namespace {

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier polls (~seconds) before giving up

template <typename T, int BG, int KW>
cudaError_t launch_bg(const CUtensorMap& map, const BwdTiledArgs& a, dim3 grid, size_t smem, cudaStream_t s) {
    auto kern = backward_tiled_kernel<T, BG, KW>;
    static size_t attr_bytes = 0;   // per instantiation; raising the limit again is harmless
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    kern<<<grid, kBwdThreads, smem, s>>>(map, a);
    return cudaGetLastError();
}

template <typename T, int KW>
cudaError_t launch_kw(int bg, const CUtensorMap& map, const BwdTiledArgs& a, dim3 grid, size_t smem, cudaStream_t s) {
    switch (bg) {
        case 4: return launch_bg<T, 4, KW>(map, a, grid, smem, s);
        case 8: return launch_bg<T, 8, KW>(map, a, grid, smem, s);
        default: return launch_bg<T, 16, KW>(map, a, grid, smem, s);
    }
}

template <typename T>
cudaError_t launch_t(int bg, int kw, const CUtensorMap& map, const BwdTiledArgs& a, dim3 grid, size_t smem,
                     cudaStream_t s) {
    return kw == 3 ? launch_kw<T, 3>(bg, map, a, grid, smem, s) : launch_kw<T, 6>(bg, map, a, grid, smem, s);
}

}  // namespace

radon_status launch_backward_tiled(const radon_geometry* g, const void* sino, void* img, radon_dtype dt, int batch,
                                   int images_per_cta, const Epilogue& ep, cudaStream_t s, std::string* why) {
    const int esz = dt == RADON_F32 ? 4 : 2;
    const int align = 16 / esz;
    // samples per candidate window: the window spans 2 (|dx|+|dy|)/h^2 <= 2 sqrt(2) / h samples
    const double span = 2.0 * std::sqrt(2.0) / g->h + 2e-4;
    const int kw_needed = (int)std::floor(span) + 1;
    if (kw_needed > 6) {
        *why = "sampling step too small for the tiled adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const int kw = kw_needed <= 3 ? 3 : 6;
    if (((uintptr_t)sino & 15) != 0) {
        *why = "sinogram pointer not 16-byte aligned";
        return RADON_ERR_UNSUPPORTED;
    }
    const int wd = ((g->bwd_window + 2) + align - 1) / align * align;   // box bytes stay a multiple of 16
    const int wdb = wd + align;
    if (wdb > 256) {
        *why = "detector window wider than a TMA box";
        return RADON_ERR_UNSUPPORTED;
    }
    const long long total = (long long)batch * g->V * g->D;
    if (total + wdb >= (1LL << 31)) {
        *why = "sinogram batch exceeds 2^31 elements";
        return RADON_ERR_UNSUPPORTED;
    }
    int bg = images_per_cta;
    if (bg == 0) bg = batch >= 16 ? 16 : (batch >= 8 ? 8 : 4);
    if (bg != 4 && bg != 8 && bg != 16) {
        *why = "images_per_cta must be 4, 8 or 16 for the tiled adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const int stage_stride = (wdb * esz + 127) / 128 * 128;
    const size_t smem = bwd_smem_bytes(bg, wd, stage_stride);
    if (smem > 227 * 1024) {
        *why = "shared memory budget exceeded";
        return RADON_ERR_UNSUPPORTED;
    }
    // The whole sinogram batch as one 1-D tensor (element x = (b V + v) D + d): per-view windows
    // need no row-stride alignment, so any detector count works.  A rank-2 description with a
    // unit outer dimension is the same layout, used if the driver refuses rank 1.
    CUtensorMap map;
    const uint64_t dims[2] = {(uint64_t)total, 1};
    const uint64_t strides[1] = {(uint64_t)((total * esz + 15) / 16 * 16)};
    const uint32_t box[2] = {(uint32_t)wdb, 1};
    int rank = 1;
    int rc = encode_tiled(&map, tma_dtype(dt), 1, const_cast<void*>(sino), dims, strides, box,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc != 0) {
        rank = 2;
        rc = encode_tiled(&map, tma_dtype(dt), 2, const_cast<void*>(sino), dims, strides, box,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    }
    if (rc != 0) {
        *why = "cuTensorMapEncodeTiled rejected the sinogram descriptor (CUresult " + std::to_string(rc) + ")";
        return RADON_ERR_UNSUPPORTED;
    }
    BwdTiledArgs a;
    a.rays = g->d_ray;
    a.nks = g->d_nk;
    a.views = g->d_view;
    a.img = img;
    a.n = g->n;
    a.V = g->V;
    a.D = g->D;
    a.B = batch;
    a.h = (float)g->h;
    a.ep = ep;
    a.wd = wd;
    a.wdb = wdb;
    a.align = align;
    a.stage_stride = stage_stride;
    a.tiles_x = (g->n + kBwdTile - 1) / kBwdTile;
    a.err = device_error_word();
    if (a.err == nullptr) {
        *why = "device error word unavailable";
        return RADON_ERR_CUDA;
    }
    const char* stall = std::getenv("RADON_TEST_STALL_TMA");
    a.stall_test = (stall != nullptr && stall[0] == '1') ? 1 : 0;
    a.spin_limit = a.stall_test ? 4096u : kSpinLimit;
    a.tma_rank = rank;
    dim3 grid((unsigned)(a.tiles_x * a.tiles_x), (unsigned)((batch + bg - 1) / bg));
    cudaError_t e;
    switch (dt) {
        case RADON_F16: e = launch_t<__half>(bg, kw, map, a, grid, smem, s); break;
        case RADON_BF16: e = launch_t<__nv_bfloat16>(bg, kw, map, a, grid, smem, s); break;
        default: e = launch_t<float>(bg, kw, map, a, grid, smem, s); break;
    }
    if (e != cudaSuccess) {
        *why = std::string("tiled adjoint launch: ") + cudaGetErrorString(e);
        return RADON_ERR_CUDA;
    }
    return RADON_OK;
}

}  // namespace radon
