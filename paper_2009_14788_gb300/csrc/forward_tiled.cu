// Host launcher and instantiations of the tiled forward projection (forward_tiled.cuh).
#include <algorithm>

#include "forward_tiled.cuh"
#include "tensor_map.h"

namespace radon {

namespace {

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier polls (~seconds) before giving up

// FP16 storage takes FP16 weights in mixed-precision FMAs only when the config asks for them and the
// epilogue adds nothing to the projection (a fused residual keeps FP32 weights); the default is FP32.
bool fp16_weights(const radon_launch_config* cfg, const Epilogue& ep) {
    return cfg != nullptr && cfg->weights == RADON_WEIGHTS_F16 && ep.add == nullptr;
}

template <typename T, int MODE>
cudaError_t launch_t(const CUtensorMap& mv, const CUtensorMap& mh, const FwdTiledArgs& a, dim3 grid, size_t smem,
                     cudaStream_t s) {
    auto kern = forward_tiled_kernel<T, MODE>;
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    kern<<<grid, kFwdThreads, smem, s>>>(mv, mh, a);
    return cudaGetLastError();
}

}  // namespace

radon_status launch_forward_tiled(radon_geometry* g, const void* img, void* sino, radon_dtype dt, int batch,
                                  const radon_launch_config* cfg, const Epilogue& ep, cudaStream_t s,
                                  std::string* why) {
    const int esz = dt == RADON_F32 ? 4 : 2;
    const int align = 16 / esz;
    const int BG = 16 / esz;
    if (g->n % align != 0) {
        *why = "image side must be a multiple of 16 bytes of storage for TMA rows";
        return RADON_ERR_UNSUPPORTED;
    }
    if (((uintptr_t)img & 15) != 0) {
        *why = "image pointer not 16-byte aligned";
        return RADON_ERR_UNSUPPORTED;
    }
    int G = cfg && cfg->views_per_cta ? cfg->views_per_cta : 4;
    if (G != 1 && G != 2 && G != 4 && G != 8) {
        *why = "views_per_cta must be 1, 2, 4 or 8 for the tiled forward";
        return RADON_ERR_UNSUPPORTED;
    }
    const int Dt = kFwdRays / G;
    const int R = cfg && cfg->rows_per_slab ? cfg->rows_per_slab : 8;
    if (R < 2 || R > 64 || (R & 1)) {
        *why = "rows_per_slab must be even and in [2, 64]";
        return RADON_ERR_UNSUPPORTED;
    }
    const int maxw = forward_band_width(g, G, Dt, R);
    const int wbox = (maxw + 2 + align - 1 + align - 1) / align * align;
    const int rbox_h = (R + align + align - 1) / align * align;   // R + 2 rows at an even offset < align
    if (wbox > 256 || rbox_h > 256) {
        *why = "working band wider than a TMA box";
        return RADON_ERR_UNSUPPORTED;
    }
    const int wc = (wbox + 7) / 8 * 8;   // row pitch = 0 (mod 8) texels: fewest shared-memory bank conflicts
    const int stage_bytes = std::max(wbox * (R + 2) * 16, rbox_h * wbox * 16);
    const size_t smem = fwd_smem_bytes(stage_bytes, R, wc);
    if (smem > 227 * 1024) {
        *why = "shared memory budget exceeded";
        return RADON_ERR_UNSUPPORTED;
    }
    int gi = 0;
    while ((1 << gi) < G) ++gi;
    const uint64_t dims[3] = {(uint64_t)g->n, (uint64_t)g->n, (uint64_t)batch};
    const uint64_t strides[2] = {(uint64_t)g->n * esz, (uint64_t)g->n * g->n * esz};
    const uint32_t box_v[3] = {(uint32_t)wbox, (uint32_t)(R + 2), (uint32_t)BG};
    const uint32_t box_h[3] = {(uint32_t)rbox_h, (uint32_t)wbox, (uint32_t)BG};
    CUtensorMap mv, mh;
    int rc = encode_tiled(&mv, tma_dtype(dt), 3, const_cast<void*>(img), dims, strides, box_v,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc == 0)
        rc = encode_tiled(&mh, tma_dtype(dt), 3, const_cast<void*>(img), dims, strides, box_h,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc != 0) {
        *why = "cuTensorMapEncodeTiled rejected the image descriptor (CUresult " + std::to_string(rc) + ")";
        return RADON_ERR_UNSUPPORTED;
    }
    FwdTiledArgs a;
    a.rays = g->d_ray;
    a.nks = g->d_nk;
    a.groups = g->d_groups + g->group_offset[gi];
    a.sino = sino;
    a.n = g->n;
    a.V = g->V;
    a.D = g->D;
    a.B = batch;
    a.h = (float)g->h;
    a.ep = ep;
    a.G = G;
    a.Dt = Dt;
    a.pair_views = G >= 2 && g->fwd_pair_views ? 1 : 0;
    a.n_dr = (g->D + Dt - 1) / Dt;
    a.R = R;
    a.n_slabs = (g->n + 4 + R - 1) / R;
    a.wbox = wbox;
    a.wc = wc;
    a.rbox_h = rbox_h;
    a.align = align;
    a.stage_bytes = stage_bytes;
    a.err = device_error_word();
    if (a.err == nullptr) {
        *why = "device error word unavailable";
        return RADON_ERR_CUDA;
    }
    a.spin_limit = kSpinLimit;
    a.stages = 2;
    a.vec_store = (g->D % 2 == 0 && ((uintptr_t)sino % (2 * esz)) == 0) ? 1 : 0;
    const long long nblk = (long long)g->group_count[gi] * a.n_dr;
    if (nblk > 0x7fffffffLL) {
        *why = "too many CTAs";
        return RADON_ERR_UNSUPPORTED;
    }
    dim3 grid((unsigned)nblk, (unsigned)((batch + BG - 1) / BG));
    cudaError_t e;
    switch (dt) {
        case RADON_F16:
            e = fp16_weights(cfg, ep) ? launch_t<__half, kMathF16W>(mv, mh, a, grid, smem, s)
                                      : launch_t<__half, kMathScalar>(mv, mh, a, grid, smem, s);
            break;
        case RADON_BF16: e = launch_t<__nv_bfloat16, kMathScalar>(mv, mh, a, grid, smem, s); break;
        default: e = launch_t<float, kMathScalar>(mv, mh, a, grid, smem, s); break;
    }
    if (e != cudaSuccess) {
        *why = std::string("tiled forward launch: ") + cudaGetErrorString(e);
        return RADON_ERR_CUDA;
    }
    return RADON_OK;
}

}  // namespace radon

namespace radon {

namespace {

template <typename T, int MODE, int NG, int LN>
cudaError_t launch_packed_ng(const CUtensorMap& mr, const CUtensorMap& mc, const FwdTiledArgs& a, dim3 grid,
                             size_t smem, cudaStream_t s) {
    auto kern = forward_packed_kernel<T, MODE, NG, LN>;
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    kern<<<grid, kFwdThreads, smem, s>>>(mr, mc, a);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_packed_t(const CUtensorMap& mr, const CUtensorMap& mc, const FwdTiledArgs& a, dim3 grid,
                            size_t smem, int NG, int LN, cudaStream_t s) {
    if (LN == 2) return launch_packed_ng<T, MODE, 1, 2>(mr, mc, a, grid, smem, s);
    return NG == 2 ? launch_packed_ng<T, MODE, 2, 1>(mr, mc, a, grid, smem, s)
                   : launch_packed_ng<T, MODE, 1, 1>(mr, mc, a, grid, smem, s);
}

}  // namespace

radon_status packed_forward_shape(radon_geometry* g, radon_dtype dt, int batch, const radon_launch_config* cfg,
                                  bool f16w, int lanes, PackedFwdShape* out, std::string* why) {
    const int esz = dt == RADON_F32 ? 4 : 2;
    const int BG = 16 / esz;
    const int G = cfg && cfg->views_per_cta ? cfg->views_per_cta : 8;
    if (G != 1 && G != 2 && G != 4 && G != 8) {
        *why = "views_per_cta must be 1, 2, 4 or 8 for the tiled forward";
        return RADON_ERR_UNSUPPORTED;
    }
    if (lanes != 1 && lanes != 2) {
        *why = "lanes per ray must be 1 or 2";
        return RADON_ERR_UNSUPPORTED;
    }
    const int Dt = kFwdRays / (G * lanes);
    // images per CTA: one texel group (BG images) or two groups sharing each sample's index work
    const int ipc = cfg ? cfg->images_per_cta : 0;
    if (ipc != 0 && ipc != BG && ipc != 2 * BG) {
        *why = "images_per_cta must be 0, " + std::to_string(BG) + " or " + std::to_string(2 * BG) +
               " for the packed forward";
        return RADON_ERR_UNSUPPORTED;
    }
    if (lanes == 2 && ipc == 2 * BG) {
        *why = "two lanes per ray take one texel group";
        return RADON_ERR_UNSUPPORTED;
    }
    // Default: 16-bit batches of more than one group pair their groups (one sample's index and weight
    // work then serves 16 images; measured 7-9 % faster on the fan and parallel workloads); FP32
    // texels (4 images each) measured slower paired.  Rows per slab: 16 for one group; 14 for two
    // (2 CTAs/SM), 8 with FP16 weights (3 CTAs/SM), the fastest of 8-16 rows measured.  A default pair
    // whose buffers would not fit falls back to one group.
    int NG = lanes == 2 ? 1 : ipc != 0 ? (ipc == 2 * BG ? 2 : 1) : (esz == 2 && batch > BG ? 2 : 1);
    for (;;) {
        const int R = cfg && cfg->rows_per_slab ? cfg->rows_per_slab : (NG == 2 ? (f16w ? 8 : 14) : 16);
        if (R < 2 || R > 64 || (R & 1)) {
            *why = "rows_per_slab must be even and in [2, 64]";
            return RADON_ERR_UNSUPPORTED;
        }
        const int maxw = forward_band_width(g, G, Dt, R);
        const int wbox = (maxw + 2 + 7) / 8 * 8;   // row pitch = 0 (mod 8) texels: fewest bank conflicts (measured)
        if (wbox > 256) {
            *why = "working band wider than a TMA box";
            return RADON_ERR_UNSUPPORTED;
        }
        // As many ring stages (up to 4) as keep three CTAs resident per SM (3 x (smem + 1 KB) <= 228 KB).
        int stages = 2;
        while (stages < kFwdMaxStages && fwd_packed_smem_bytes(R, wbox, stages + 1, NG) <= 75 * 1024) ++stages;
        const size_t smem = fwd_packed_smem_bytes(R, wbox, stages, NG);
        if (smem <= 227 * 1024) {
            *out = PackedFwdShape{G, Dt, NG, lanes, R, wbox, stages, smem};
            return RADON_OK;
        }
        if (ipc == 0 && NG == 2) {
            NG = 1;
            continue;
        }
        *why = "shared memory budget exceeded";
        return RADON_ERR_UNSUPPORTED;
    }
}

radon_status launch_forward_packed(radon_geometry* g, const void* packed, void* sino, radon_dtype dt, int batch,
                                   const radon_launch_config* cfg, const Epilogue& ep, cudaStream_t s,
                                   std::string* why, int lanes) {
    const int esz = dt == RADON_F32 ? 4 : 2;
    const int BG = 16 / esz;
    if (((uintptr_t)packed & 15) != 0) {
        *why = "workspace not 16-byte aligned";
        return RADON_ERR_UNSUPPORTED;
    }
    PackedFwdShape sh;
    const radon_status st =
        packed_forward_shape(g, dt, batch, cfg, dt == RADON_F16 && fp16_weights(cfg, ep), lanes, &sh, why);
    if (st != RADON_OK) return st;
    const int G = sh.G, Dt = sh.Dt, NG = sh.NG, LN = sh.LN, R = sh.R, wbox = sh.wbox, stages = sh.stages;
    const size_t smem = sh.smem;
    int gi = 0;
    while ((1 << gi) < G) ++gi;
    const int groups = (batch + BG - 1) / BG;
    const uint64_t n = (uint64_t)g->n;
    const uint64_t dims[4] = {(uint64_t)BG, n, n, (uint64_t)groups};
    const uint64_t strides[3] = {16, n * 16, n * n * 16};
    const uint32_t box[4] = {(uint32_t)BG, (uint32_t)wbox, (uint32_t)(R + 2), (uint32_t)NG};
    const unsigned char* rows = reinterpret_cast<const unsigned char*>(packed);
    const unsigned char* cols = rows + (size_t)groups * n * n * 16;
    CUtensorMap mr, mc;
    int rc = encode_tiled(&mr, tma_dtype(dt), 4, const_cast<unsigned char*>(rows), dims, strides, box,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc == 0)
        rc = encode_tiled(&mc, tma_dtype(dt), 4, const_cast<unsigned char*>(cols), dims, strides, box,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc != 0) {
        *why = "cuTensorMapEncodeTiled rejected the packed-image descriptor (CUresult " + std::to_string(rc) + ")";
        return RADON_ERR_UNSUPPORTED;
    }
    FwdTiledArgs a;
    a.rays = g->d_ray;
    a.nks = g->d_nk;
    a.groups = g->d_groups + g->group_offset[gi];
    a.sino = sino;
    a.n = g->n;
    a.V = g->V;
    a.D = g->D;
    a.B = batch;
    a.h = (float)g->h;
    a.ep = ep;
    a.G = G;
    a.Dt = Dt;
    a.pair_views = LN == 1 && G >= 2 && g->fwd_pair_views ? 1 : 0;
    a.n_dr = (g->D + Dt - 1) / Dt;
    a.R = R;
    a.n_slabs = (g->n + 4 + R - 1) / R;
    a.wbox = wbox;
    a.wc = wbox;
    a.rbox_h = 0;
    a.align = 1;
    a.stage_bytes = 0;
    a.err = device_error_word();
    if (a.err == nullptr) {
        *why = "device error word unavailable";
        return RADON_ERR_CUDA;
    }
    a.spin_limit = kSpinLimit;
    a.stages = stages;
    a.vec_store = (g->D % 2 == 0 && ((uintptr_t)sino % (2 * esz)) == 0) ? 1 : 0;
    const long long nblk = (long long)g->group_count[gi] * a.n_dr;
    dim3 grid((unsigned)nblk, (unsigned)((groups + NG - 1) / NG));
    cudaError_t e;
    switch (dt) {
        case RADON_F16:
            e = fp16_weights(cfg, ep) ? launch_packed_t<__half, kMathF16W>(mr, mc, a, grid, smem, NG, LN, s)
                                      : launch_packed_t<__half, kMathScalar>(mr, mc, a, grid, smem, NG, LN, s);
            break;
        case RADON_BF16: e = launch_packed_t<__nv_bfloat16, kMathScalar>(mr, mc, a, grid, smem, NG, LN, s); break;
        default: e = launch_packed_t<float, kMathScalar>(mr, mc, a, grid, smem, NG, LN, s); break;
    }
    if (e != cudaSuccess) {
        *why = std::string("packed forward launch: ") + cudaGetErrorString(e);
        return RADON_ERR_CUDA;
    }
    return RADON_OK;
}

}  // namespace radon
