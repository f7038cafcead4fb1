// Pixel-driven interpolating backprojector (the kind the paper's comparisons use, Section 3.1).
//
// For every pixel and view: the pixel centre's continuous detector index t from the view's projective
// detector map (the same map that bounds the exact adjoint's windows), the sinogram row linearly
// interpolated there (bins outside [0, D) read as zero), weighted by the ray density |grad t| (bins
// per pixel: 1 / ds for parallel beams) so that the result approximates the exact adjoint.  One
// thread per pixel, 8 images per CTA sharing each view's coordinate and weights; sinogram rows read
// through L1 (a warp's pixels touch a few dozen neighbouring bins).
#include "dtype.cuh"
#include "radon_internal.h"

namespace radon {

namespace {

constexpr int kIbpImages = 8;
constexpr int kIbpTile = 16;

template <typename T>
__global__ void __launch_bounds__(kIbpTile * kIbpTile) interp_bp_kernel(const T* __restrict__ sino, T* __restrict__ img,
                                                                        const ViewF* __restrict__ views, int n, int V,
                                                                        int D, int B, int tiles_x) {
    const int ti = (blockIdx.x / tiles_x) * kIbpTile, tj = (blockIdx.x % tiles_x) * kIbpTile;
    const int i = ti + threadIdx.x / kIbpTile, j = tj + threadIdx.x % kIbpTile;
    if (i >= n || j >= n) return;
    const int b0 = blockIdx.y * kIbpImages;
    const int nb = min(kIbpImages, B - b0);
    const float x = (float)j, y = (float)i;
    const long long vd = (long long)V * D;
    float acc[kIbpImages];
#pragma unroll
    for (int b = 0; b < kIbpImages; ++b) acc[b] = 0.0f;
    for (int v = 0; v < V; ++v) {
        const ViewF vf = views[v];
        const float den = fmaf(vf.bx, x, fmaf(vf.by, y, vf.b0));
        const float t = fmaf(vf.ax, x, fmaf(vf.ay, y, vf.a0)) / den;   // IEEE: t is needed to ~1e-5 bins
        const float gx = fmaf(-t, vf.bx, vf.ax), gy = fmaf(-t, vf.by, vf.ay);
        const float w = sqrtf(fmaf(gx, gx, gy * gy)) / fabsf(den);
        const float fl = floorf(t);
        const float f = t - fl;
        const int k = (int)fl;
        const bool in0 = k >= 0 && k < D, in1 = k + 1 >= 0 && k + 1 < D;
        const float w0 = w * (1.0f - f), w1 = w * f;
        const T* row = sino + (long long)b0 * vd + (long long)v * D;
#pragma unroll
        for (int b = 0; b < kIbpImages; ++b) {
            if (b < nb) {
                const float y0 = in0 ? load_f32(row + (long long)b * vd + k) : 0.0f;
                const float y1 = in1 ? load_f32(row + (long long)b * vd + k + 1) : 0.0f;
                acc[b] = fmaf(w0, y0, fmaf(w1, y1, acc[b]));
            }
        }
    }
    const long long npix = (long long)n * n;
#pragma unroll
    for (int b = 0; b < kIbpImages; ++b)
        if (b < nb) img[(long long)(b0 + b) * npix + (long long)i * n + j] = from_f32<T>(acc[b]);
}

}  // namespace

}  // namespace radon

using namespace radon;

extern "C" RADON_API radon_status radon_backproject_interpolating(const radon_geometry* g, const void* sino, void* img,
                                                                  radon_dtype dtype, int batch, void* stream) {
    radon_status st = validate_call(g, sino, img, dtype, batch);
    if (st != RADON_OK) return st;
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (batch == 0) return RADON_OK;
    st = check_device(g);
    if (st != RADON_OK) return st;
    const int tiles_x = (g->n + kIbpTile - 1) / kIbpTile;
    const long long tiles = (long long)tiles_x * tiles_x;
    const long long groups = (batch + kIbpImages - 1) / kIbpImages;
    if (tiles > 0x7fffffffLL || groups > 65535) return fail(RADON_ERR_UNSUPPORTED, "image or batch too large");
    const dim3 grid((unsigned)tiles, (unsigned)groups);
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
        case RADON_F16:
            interp_bp_kernel<__half><<<grid, kIbpTile * kIbpTile, 0, s>>>((const __half*)sino, (__half*)img, g->d_view,
                                                                         g->n, g->V, g->D, batch, tiles_x);
            break;
        case RADON_BF16:
            interp_bp_kernel<__nv_bfloat16><<<grid, kIbpTile * kIbpTile, 0, s>>>(
                (const __nv_bfloat16*)sino, (__nv_bfloat16*)img, g->d_view, g->n, g->V, g->D, batch, tiles_x);
            break;
        default:
            interp_bp_kernel<float><<<grid, kIbpTile * kIbpTile, 0, s>>>((const float*)sino, (float*)img, g->d_view,
                                                                        g->n, g->V, g->D, batch, tiles_x);
            break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "interpolating backprojection launch");
    count_launches(1);
    return RADON_OK;
}

extern "C" RADON_API radon_status radon_backproject_interpolating_ws(const radon_geometry* g, const void* sino, void* img,
                                                                     radon_dtype dtype, int batch, void* workspace,
                                                                     size_t workspace_bytes, void* stream) {
    radon_status st = validate_call(g, sino, img, dtype, batch);
    if (st != RADON_OK) return st;
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (workspace != nullptr && ((uintptr_t)workspace & 15) != 0)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    if (batch == 0) return RADON_OK;
    st = check_device(g);
    if (st != RADON_OK) return st;
    const int bg = backward_packed_images_per_cta(g, batch, dtype, nullptr);
    if (workspace != nullptr && workspace_bytes >= packed_sino_bytes(g->V, g->D, batch, bg, dtype)) {
        cudaStream_t s = (cudaStream_t)stream;
        cudaError_t e = launch_pack_sino(sino, workspace, g->V, g->D, batch, bg, dtype, s);
        if (e != cudaSuccess) return cuda_fail(e, "sinogram pack launch");
        count_launches(1);
        std::string why;
        st = launch_backward_packed(g, workspace, img, dtype, batch, bg, identity_epilogue(), s, &why, true);
        if (st == RADON_OK) {
            count_launches(1);
            return RADON_OK;
        }
        if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
    }
    return radon_backproject_interpolating(g, sino, img, dtype, batch, stream);
}
