// Plain projector kernels: one thread per ray (forward), one thread per pixel (adjoint),
// operands read straight from global memory through the read-only cache.  They are the
// simple comparison form of the operator and the fallback for any shape the tiled kernels
// do not take.  Arithmetic is FP32 for every storage type.
#include <cmath>

#include "dtype.cuh"
#include "epilogue.cuh"
#include "radon_internal.h"

namespace radon {

namespace {

// Samples are processed in chunks of kChunk; each chunk re-bases its start position from the
// split-precision table (integer base + small fraction), so the FP32 position error stays at a
// few 1e-6 pixels however far the sample lies from the image origin.
constexpr int kChunk = 32;

// Forward: y[b][v][d] = h * sum_k bilinear(x_b, sample k of ray (v, d)).
template <typename T>
__global__ void forward_plain_kernel(const T* __restrict__ img, T* __restrict__ sino, const RayT* __restrict__ rays,
                                     const int* __restrict__ nks, int n, int64_t rays_per_image, int64_t total,
                                     float h, const Epilogue ep) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t b = idx / rays_per_image;
    const int64_t r = idx - b * rays_per_image;
    const RayT ray = rays[r];
    const int nk = nks[r];
    const float dx = ray.dxh + ray.dxl, dy = ray.dyh + ray.dyl;
    const T* x = img + b * (int64_t)n * n;
    float acc = 0.0f;
    for (int kb = 0; kb < nk; kb += kChunk) {
        const float kbf = (float)kb;
        const float qx = kbf * ray.dxh, qy = kbf * ray.dyh;   // exact products
        const float Qx = floorf(qx), Qy = floorf(qy);
        const float sx = fmaf(kbf, ray.dxl, ray.fx0 + (qx - Qx));
        const float sy = fmaf(kbf, ray.dyl, ray.fy0 + (qy - Qy));
        const int jb = ray.J0 + (int)Qx, ib = ray.I0 + (int)Qy;
        const int kend = min(nk - kb, kChunk);
        for (int kk = 0; kk < kend; ++kk) {
            const float lx = fmaf((float)kk, dx, sx);
            const float ly = fmaf((float)kk, dy, sy);
            const float flx = floorf(lx), fly = floorf(ly);
            const float a = lx - flx, c = ly - fly;
            const int j = jb + (int)flx, i = ib + (int)fly;
            const bool j0in = j >= 0 && j < n, j1in = j + 1 >= 0 && j + 1 < n;
            const bool i0in = i >= 0 && i < n, i1in = i + 1 >= 0 && i + 1 < n;
            const int64_t base = (int64_t)i * n + j;
            const float v00 = (i0in && j0in) ? load_f32(x + base) : 0.0f;
            const float v01 = (i0in && j1in) ? load_f32(x + base + 1) : 0.0f;
            const float v10 = (i1in && j0in) ? load_f32(x + base + n) : 0.0f;
            const float v11 = (i1in && j1in) ? load_f32(x + base + n + 1) : 0.0f;
            acc += (1.0f - c) * ((1.0f - a) * v00 + a * v01) + c * ((1.0f - a) * v10 + a * v11);
        }
    }
    sino[idx] = from_f32<T>(epilogue_value<T>(ep, h * acc, idx));
}

__device__ __forceinline__ float det_coord(const ViewF& vf, float x, float y) {
    return fmaf(vf.ax, x, fmaf(vf.ay, y, vf.a0)) / fmaf(vf.bx, x, fmaf(vf.by, y, vf.b0));
}

// Adjoint (gather): x[b][i][j] = h * sum_v sum_d y[b][v][d] * sum_k w_k(i, j), where w_k is the
// bilinear weight of sample k of ray (v, d) on pixel (i, j).  Candidate rays are those whose
// detector index lies between the projections of the pixel's 2x2 support square; candidate
// samples lie within (|dx|+|dy|)/|step|^2 of the ray's closest approach.  Extra candidates
// contribute exactly zero, so the windows only need to be wide enough.  The first candidate's
// offset from the pixel is re-based from the split-precision table.
template <typename T>
__global__ void backward_plain_kernel(const T* __restrict__ sino, T* __restrict__ img, const RayT* __restrict__ rays,
                                      const int* __restrict__ nks, const ViewF* __restrict__ views, int n, int V,
                                      int D, int64_t total, float h, const Epilogue ep) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t npix = (int64_t)n * n;
    const int64_t b = idx / npix;
    const int64_t p = idx - b * npix;
    const int i = (int)(p / n), j = (int)(p - (int64_t)(p / n) * n);
    const float xf = (float)j, yf = (float)i;
    const T* y = sino + b * (int64_t)V * D;
    const float eps = 1e-3f;
    float acc = 0.0f;
    for (int v = 0; v < V; ++v) {
        const ViewF vf = views[v];
        const float t0 = det_coord(vf, xf - 1.0f, yf - 1.0f);
        const float t1 = det_coord(vf, xf + 1.0f, yf - 1.0f);
        const float t2 = det_coord(vf, xf - 1.0f, yf + 1.0f);
        const float t3 = det_coord(vf, xf + 1.0f, yf + 1.0f);
        const float tmin = fminf(fminf(t0, t1), fminf(t2, t3));
        const float tmax = fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
        const int d0 = (int)fmaxf(0.0f, ceilf(tmin - eps));
        const int d1 = (int)fminf((float)(D - 1), floorf(tmax + eps));
        for (int d = d0; d <= d1; ++d) {
            const int64_t r = (int64_t)v * D + d;
            const int nk = nks[r];
            if (nk == 0) continue;
            const RayT ray = rays[r];
            const float dx = ray.dxh + ray.dxl, dy = ray.dyh + ray.dyl;
            const float ex = (float)(j - ray.J0) - ray.fx0, ey = (float)(i - ray.I0) - ray.fy0;
            const float il = 1.0f / fmaf(dx, dx, dy * dy);
            const float kc = fmaf(ex, dx, ey * dy) * il;
            const float kr = (fabsf(dx) + fabsf(dy)) * il;
            const int k0 = (int)fmaxf(0.0f, ceilf(kc - kr - eps));
            const int k1 = (int)fminf((float)(nk - 1), floorf(kc + kr + eps));
            if (k0 > k1) continue;
            const float k0f = (float)k0;
            const float qx = k0f * ray.dxh, qy = k0f * ray.dyh;   // exact products
            const float Qx = floorf(qx), Qy = floorf(qy);
            float rx = ((float)(ray.J0 - j) + Qx) + fmaf(k0f, ray.dxl, ray.fx0 + (qx - Qx));
            float ry = ((float)(ray.I0 - i) + Qy) + fmaf(k0f, ray.dyl, ray.fy0 + (qy - Qy));
            float w = 0.0f;
            for (int k = k0; k <= k1; ++k) {
                const float wx = fmaxf(0.0f, 1.0f - fabsf(rx));
                const float wy = fmaxf(0.0f, 1.0f - fabsf(ry));
                w = fmaf(wx, wy, w);
                rx += dx;
                ry += dy;
            }
            if (w != 0.0f) acc = fmaf(w, load_f32(y + r), acc);
        }
    }
    img[idx] = from_f32<T>(epilogue_value<T>(ep, h * acc, idx));
}

template <typename T>
cudaError_t forward_plain_t(const radon_geometry* g, const void* img, void* sino, int batch, int threads,
                            const Epilogue& ep, cudaStream_t s) {
    const int64_t rays = (int64_t)g->V * g->D;
    const int64_t total = rays * batch;
    if (total == 0) return cudaSuccess;
    const int64_t blocks = (total + threads - 1) / threads;
    forward_plain_kernel<T><<<(unsigned)blocks, threads, 0, s>>>((const T*)img, (T*)sino, g->d_ray, g->d_nk, g->n,
                                                                 rays, total, (float)g->h, ep);
    return cudaGetLastError();
}

template <typename T>
cudaError_t backward_plain_t(const radon_geometry* g, const void* sino, void* img, int batch, int threads,
                             const Epilogue& ep, cudaStream_t s) {
    const int64_t total = (int64_t)g->n * g->n * batch;
    if (total == 0) return cudaSuccess;
    const int64_t blocks = (total + threads - 1) / threads;
    backward_plain_kernel<T><<<(unsigned)blocks, threads, 0, s>>>((const T*)sino, (T*)img, g->d_ray, g->d_nk,
                                                                  g->d_view, g->n, g->V, g->D, total, (float)g->h,
                                                                  ep);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward_plain(const radon_geometry* g, const void* img, void* sino, radon_dtype dt, int batch,
                                 int threads, const Epilogue& ep, cudaStream_t s) {
    if (threads <= 0) threads = 256;
    switch (dt) {
        case RADON_F32: return forward_plain_t<float>(g, img, sino, batch, threads, ep, s);
        case RADON_F16: return forward_plain_t<__half>(g, img, sino, batch, threads, ep, s);
        case RADON_BF16: return forward_plain_t<__nv_bfloat16>(g, img, sino, batch, threads, ep, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_backward_plain(const radon_geometry* g, const void* sino, void* img, radon_dtype dt, int batch,
                                  int threads, const Epilogue& ep, cudaStream_t s) {
    if (threads <= 0) threads = 256;
    switch (dt) {
        case RADON_F32: return backward_plain_t<float>(g, sino, img, batch, threads, ep, s);
        case RADON_F16: return backward_plain_t<__half>(g, sino, img, batch, threads, ep, s);
        case RADON_BF16: return backward_plain_t<__nv_bfloat16>(g, sino, img, batch, threads, ep, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace radon
