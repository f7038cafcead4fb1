// Host dispatch of the packed adjoint (backward_packed.cuh): image-group size, ring descriptor of
// the ray table, and the launcher instantiated for the storage type.
#include <cmath>

#include "backward_packed.cuh"

namespace radon {

#define RADON_BWDP_EXTERN(T, BG)                                                                              \
    extern template radon_status launch_backward_packed_t<T, BG>(const radon_geometry*, const void*, void*,       \
                                                                 radon_dtype, int, int, const Epilogue&,          \
                                                                 cudaStream_t, std::string*, const CUtensorMap&, \
                                                                 uint32_t, int*);
RADON_BWDP_EXTERN(float, 8)
RADON_BWDP_EXTERN(float, 16)
RADON_BWDP_EXTERN(float, 32)
RADON_BWDP_EXTERN(__half, 8)
RADON_BWDP_EXTERN(__half, 16)
RADON_BWDP_EXTERN(__half, 32)
RADON_BWDP_EXTERN(__nv_bfloat16, 8)
RADON_BWDP_EXTERN(__nv_bfloat16, 16)
RADON_BWDP_EXTERN(__nv_bfloat16, 32)
#undef RADON_BWDP_EXTERN

namespace {

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier polls (~seconds) before giving up

template <typename T>
radon_status launch_bg(const radon_geometry* g, const void* packed, void* img, radon_dtype dt, int batch, int bg,
                       int kw, const Epilogue& ep, cudaStream_t s, std::string* why, const CUtensorMap& rmap, int* err) {
    switch (bg) {
        case 8: return launch_backward_packed_t<T, 8>(g, packed, img, dt, batch, kw, ep, s, why, rmap, kSpinLimit, err);
        case 16: return launch_backward_packed_t<T, 16>(g, packed, img, dt, batch, kw, ep, s, why, rmap, kSpinLimit, err);
        default: return launch_backward_packed_t<T, 32>(g, packed, img, dt, batch, kw, ep, s, why, rmap, kSpinLimit, err);
    }
}

size_t smem_32(const radon_geometry* g, radon_dtype dt) {
    int st = 0;
    const int wd = g->bwd_window + 2;
    switch (dt) {
        case RADON_F16: return bwdp_plan<__half, 32>(wd, true, &st);
        case RADON_BF16: return bwdp_plan<__nv_bfloat16, 32>(wd, true, &st);
        default: return bwdp_plan<float, 32>(wd, true, &st);
    }
}

}  // namespace

int backward_packed_images_per_cta(const radon_geometry* g, int batch, radon_dtype dt, const radon_launch_config* cfg) {
    if (cfg != nullptr && cfg->images_per_cta != 0) return cfg->images_per_cta;
    if (batch <= 8) return 8;
    if (batch <= 16) return 16;
    // with the geometry's weight table 16-bit 16-image groups read their weights, which measured faster
    // than 32-image groups computing them (parallel 32 x 512^2, 512 views, FP16 adjoint: 1.84 vs 1.94
    // ms; FP32 rows measured no faster: a step of 4.32 vs 4.27 ms)
    if (g->d_tab_w != nullptr && dt != RADON_F32) return 16;
    // A 32-image CTA costs ~1.56x a 16-image one (each weight serves twice the images; two CTAs per
    // SM): take it when its groups cost less and its staging fits one CTA's shared memory.
    const long long g32 = (batch + 31) / 32, g16 = (batch + 15) / 16;
    if (25 * g32 < 16 * g16 && smem_32(g, dt) <= 227 * 1024) return 32;
    return 16;
}

radon_status launch_backward_packed(const radon_geometry* g, const void* packed, void* img, radon_dtype dt, int batch,
                                    int bg, const Epilogue& ep, cudaStream_t s, std::string* why, bool interpolating) {
    if (bg != 8 && bg != 16 && bg != 32) {
        *why = "images_per_cta must be 8, 16 or 32 for the packed adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    if (((uintptr_t)packed & 15) != 0) {
        *why = "workspace not 16-byte aligned";
        return RADON_ERR_UNSUPPORTED;
    }
    // samples per candidate window: the window spans 2 (|dx| + |dy|) / h^2 <= 2 sqrt(2) / h samples
    const double span = 2.0 * std::sqrt(2.0) / g->h + 2e-4;
    const int kw_needed = (int)std::floor(span) + 1;
    if (!interpolating && kw_needed > 6) {
        *why = "sampling step too small for the tiled adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const int kw = interpolating ? 0 : (kw_needed <= 3 ? 3 : 6);
    const int wd = g->bwd_window + 2;
    if (wd > 256) {
        *why = "detector window wider than a TMA box";
        return RADON_ERR_UNSUPPORTED;
    }
    // the ray table as rows of 8 words (bit copies), one row per ray, rays of view v at v * D
    CUtensorMap rmap;
    const uint64_t rdims[2] = {8, (uint64_t)g->V * g->D};
    const uint64_t rstrides[1] = {32};
    const uint32_t rbox[2] = {8, (uint32_t)wd};
    const int rc = encode_tiled(&rmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g->d_ray, rdims, rstrides, rbox,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc != 0) {
        *why = "cuTensorMapEncodeTiled rejected the ray-table descriptor (CUresult " + std::to_string(rc) + ")";
        return RADON_ERR_UNSUPPORTED;
    }
    int* err = device_error_word();
    if (err == nullptr) {
        *why = "device error word unavailable";
        return RADON_ERR_CUDA;
    }
    switch (dt) {
        case RADON_F16: return launch_bg<__half>(g, packed, img, dt, batch, bg, kw, ep, s, why, rmap, err);
        case RADON_BF16: return launch_bg<__nv_bfloat16>(g, packed, img, dt, batch, bg, kw, ep, s, why, rmap, err);
        default: return launch_bg<float>(g, packed, img, dt, batch, bg, kw, ep, s, why, rmap, err);
    }
}

size_t adjoint_table_bytes(const radon_geometry* g) {
    const size_t tiles_x = (size_t)(g->n + kBwdTile - 1) / kBwdTile;
    return tiles_x * tiles_x * (size_t)g->V * (kBwdTabPairs * (2 * sizeof(float4) + sizeof(float2) + sizeof(int)) + sizeof(int));
}

void free_adjoint_table(radon_geometry* g) {
    if (g->d_tab_w) cudaFree(g->d_tab_w);
    if (g->d_tab_w5) cudaFree(g->d_tab_w5);
    if (g->d_tab_la) cudaFree(g->d_tab_la);
    if (g->d_tab_vflag) cudaFree(g->d_tab_vflag);
    g->d_tab_vflag = nullptr;
    g->d_tab_w = nullptr;
    g->d_tab_w5 = nullptr;
    g->d_tab_la = nullptr;
    g->tab_kw = 0;
    g->tab_wd = 0;
    g->tab_bytes = 0;
    g->tab_overflow = 0.0;
}

// Builds the geometry's weight table on the current device (the geometry's), synchronising it.
radon_status build_adjoint_table(radon_geometry* g, std::string* why) {
    const double span = 2.0 * std::sqrt(2.0) / g->h + 2e-4;
    const int kw_needed = (int)std::floor(span) + 1;
    if (kw_needed > 6) {
        *why = "sampling step too small for the packed adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const int kw = kw_needed <= 3 ? 3 : 6;
    const int wd = g->bwd_window + 2;
    if (wd > 256) {
        *why = "detector window wider than a TMA box";
        return RADON_ERR_UNSUPPORTED;
    }
    free_adjoint_table(g);
    const int tiles_x = (g->n + kBwdTile - 1) / kBwdTile;
    const size_t recs = (size_t)tiles_x * tiles_x * (size_t)g->V * kBwdTabPairs;
    float4* w = nullptr;
    float2* w5 = nullptr;
    int* la = nullptr;
    int* vflag = nullptr;
    unsigned long long* over = nullptr;
    const size_t tv = (size_t)tiles_x * tiles_x * (size_t)g->V;
    if (cudaMalloc(&w, recs * 2 * sizeof(float4)) != cudaSuccess || cudaMalloc(&w5, recs * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&la, recs * sizeof(int)) != cudaSuccess || cudaMalloc(&vflag, tv * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&over, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w);
        cudaFree(w5);
        cudaFree(la);
        cudaFree(vflag);
        cudaFree(over);
        *why = "device allocation of the weight table failed";
        return RADON_ERR_OOM;
    }
    constexpr int kViewsPerBlock = 16;
    cudaError_t e = cudaMemset(over, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(vflag, 0, tv * sizeof(int));
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)(tiles_x * tiles_x), (unsigned)((g->V + kViewsPerBlock - 1) / kViewsPerBlock));
        const float ih2 = (float)(1.0 / (g->h * g->h));
        if (kw == 3)
            bwdp_table_kernel<3><<<grid, kBwdTabPairs>>>(g->d_ray, g->d_view, g->n, g->V, g->D, ih2, wd, tiles_x,
                                                         kViewsPerBlock, w, w5, la, vflag, over);
        else
            bwdp_table_kernel<6><<<grid, kBwdTabPairs>>>(g->d_ray, g->d_view, g->n, g->V, g->D, ih2, wd, tiles_x,
                                                         kViewsPerBlock, w, w5, la, vflag, over);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    unsigned long long n_over = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n_over, over, sizeof(n_over), cudaMemcpyDeviceToHost);
    cudaFree(over);
    if (e != cudaSuccess) {
        cudaFree(w);
        cudaFree(w5);
        cudaFree(la);
        cudaFree(vflag);
        *why = std::string("weight table build: ") + cudaGetErrorString(e);
        return RADON_ERR_CUDA;
    }
    count_launches(1);
    g->d_tab_w = w;
    g->d_tab_w5 = w5;
    g->d_tab_la = la;
    g->d_tab_vflag = vflag;
    g->tab_kw = kw;
    g->tab_wd = wd;
    g->tab_bytes = adjoint_table_bytes(g);
    g->tab_overflow = (double)n_over / (double)recs;
    return RADON_OK;
}

}  // namespace radon
