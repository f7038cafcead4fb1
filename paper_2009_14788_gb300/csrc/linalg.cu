// Vector kernels of the iterative reconstruction (Section 4.2: Landweber iteration with its step
// size from the power method): a deterministic inner product, a scaled add / cast, and the power
// iteration itself, sequenced on the device so that the eigenvalue estimate never leaves it.
#include <algorithm>
#include <cmath>
#include <string>

#include "dtype.cuh"
#include "radon_internal.h"

namespace radon {

namespace {

constexpr int kDotBlocks = 304;    // two blocks per SM on 152 SMs
constexpr int kDotThreads = 256;
constexpr int kAxpbyThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block in a fixed order (lane tree within warps, then the warps' sums by warp 0).
__device__ double block_sum(double v) {
    __shared__ double warp_part[kDotThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < kDotThreads / 32 ? warp_part[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;   // valid in thread 0
}

// Blocks per item of a batched inner product: 304 for one item (two per SM), fewer per item for
// larger batches, at least 8.
int dot_blocks(int batch) { return batch <= 1 ? kDotBlocks : (kDotBlocks / batch > 8 ? kDotBlocks / batch : 8); }

// Stage 1: block (b, i) sums the products of a grid-stride slice of item i (FP32 per thread, FP64
// across threads).
template <typename T>
__global__ void __launch_bounds__(kDotThreads) dot_partial_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                                  long long count, double* __restrict__ partial) {
    const long long off = (long long)blockIdx.y * count;
    float s = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        s = fmaf(to_f32(a[off + i]), to_f32(b[off + i]), s);
    const double t = block_sum((double)s);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Stage 2: one block per item adds its partials in index order.
__global__ void __launch_bounds__(kDotThreads) dot_final_kernel(const double* __restrict__ partial, int n, float scale,
                                                                float* result, int accumulate) {
    const double* pp = partial + (size_t)blockIdx.x * n;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += pp[i];
    const double t = block_sum(s);
    if (threadIdx.x == 0) {
        const float v = (float)((double)scale * t);
        result[blockIdx.x] = accumulate ? result[blockIdx.x] + v : v;
    }
}

// y_i = alpha s_i x_i + beta t_i y_i over `batch` items of `count` elements; s_i = alpha_dev[i] or 1,
// t_i = beta_dev[i] or 1; y is not read when beta == 0 and beta_dev is NULL.
template <typename TX, typename TY>
__global__ void __launch_bounds__(kAxpbyThreads) axpby_kernel(const TX* __restrict__ x, TY* y, long long count,
                                                              long long total, float alpha, const float* alpha_dev,
                                                              float beta, const float* beta_dev) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool read_y = beta != 0.0f || beta_dev != nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long long item = i / count;
        const float a = alpha_dev != nullptr ? alpha * alpha_dev[item] : alpha;
        float v = a * to_f32(x[i]);
        if (read_y) v = fmaf(beta_dev != nullptr ? beta * beta_dev[item] : beta, to_f32(y[i]), v);
        y[i] = from_f32<TY>(v);
    }
}

// out[i] = num[i] / den[i] where den[i] > 0, else 0: the step lengths of the conjugate gradient
// recursions (a zero denominator means the direction or the residual has vanished).
__global__ void safe_divide_kernel(const float* num, const float* den, float* out, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch) out[i] = den[i] > 0.0f ? num[i] / den[i] : 0.0f;
}

// dst = 1 / sqrt(src) (one thread): the normalising factor of a power-method iterate.
__global__ void rsqrt_kernel(const float* src, float* dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = 1.0f / sqrtf(*src);
}

// dst = 1 / src (one thread): Landweber's step from the eigenvalue estimate.
__global__ void reciprocal_kernel(const float* src, float* dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = 1.0f / *src;
}

size_t esize(radon_dtype dt) { return dt == RADON_F32 ? 4 : 2; }

bool valid_dtype(radon_dtype dt) { return dt == RADON_F32 || dt == RADON_F16 || dt == RADON_BF16; }

template <typename TX>
cudaError_t axpby_y(const void* x, void* y, radon_dtype yt, long long count, long long total, float alpha,
                    const float* alpha_dev, float beta, const float* beta_dev, unsigned blocks, cudaStream_t s) {
    switch (yt) {
        case RADON_F32:
            axpby_kernel<TX, float><<<blocks, kAxpbyThreads, 0, s>>>((const TX*)x, (float*)y, count, total, alpha,
                                                                     alpha_dev, beta, beta_dev);
            break;
        case RADON_F16:
            axpby_kernel<TX, __half><<<blocks, kAxpbyThreads, 0, s>>>((const TX*)x, (__half*)y, count, total, alpha,
                                                                      alpha_dev, beta, beta_dev);
            break;
        default:
            axpby_kernel<TX, __nv_bfloat16><<<blocks, kAxpbyThreads, 0, s>>>((const TX*)x, (__nv_bfloat16*)y, count,
                                                                             total, alpha, alpha_dev, beta, beta_dev);
            break;
    }
    return cudaGetLastError();
}

radon_status dot_launch(const void* a, const void* b, radon_dtype dt, int batch, long long count, float scale,
                        float* result, int accumulate, double* partial, cudaStream_t s) {
    const dim3 grid((unsigned)dot_blocks(batch), (unsigned)batch);
    switch (dt) {
        case RADON_F32:
            dot_partial_kernel<float><<<grid, kDotThreads, 0, s>>>((const float*)a, (const float*)b, count, partial);
            break;
        case RADON_F16:
            dot_partial_kernel<__half><<<grid, kDotThreads, 0, s>>>((const __half*)a, (const __half*)b, count, partial);
            break;
        default:
            dot_partial_kernel<__nv_bfloat16><<<grid, kDotThreads, 0, s>>>(
                (const __nv_bfloat16*)a, (const __nv_bfloat16*)b, count, partial);
            break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dot launch");
    dot_final_kernel<<<(unsigned)batch, kDotThreads, 0, s>>>(partial, dot_blocks(batch), scale, result, accumulate);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dot launch");
    count_launches(2);
    return RADON_OK;
}

radon_status dot_launch(const void* a, const void* b, radon_dtype dt, long long count, float scale, float* result,
                        int accumulate, double* partial, cudaStream_t s) {
    return dot_launch(a, b, dt, 1, count, scale, result, accumulate, partial, s);
}

radon_status axpby_launch(const void* x, radon_dtype xt, void* y, radon_dtype yt, int batch, long long count,
                          float alpha, const float* alpha_dev, float beta, const float* beta_dev, cudaStream_t s) {
    const long long total = (long long)batch * count;
    if (total == 0) return RADON_OK;
    const long long want = (total + kAxpbyThreads - 1) / kAxpbyThreads;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    cudaError_t e;
    switch (xt) {
        case RADON_F32: e = axpby_y<float>(x, y, yt, count, total, alpha, alpha_dev, beta, beta_dev, blocks, s); break;
        case RADON_F16: e = axpby_y<__half>(x, y, yt, count, total, alpha, alpha_dev, beta, beta_dev, blocks, s); break;
        default: e = axpby_y<__nv_bfloat16>(x, y, yt, count, total, alpha, alpha_dev, beta, beta_dev, blocks, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "axpby launch");
    count_launches(1);
    return RADON_OK;
}

radon_status axpby_launch(const void* x, radon_dtype xt, void* y, radon_dtype yt, long long count, float alpha,
                          const float* alpha_dev, float beta, cudaStream_t s) {
    return axpby_launch(x, xt, y, yt, 1, count, alpha, alpha_dev, beta, nullptr, s);
}

radon_status divide_launch(const float* num, const float* den, float* out, int batch, cudaStream_t s) {
    safe_divide_kernel<<<(batch + 127) / 128, 128, 0, s>>>(num, den, out, batch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "divide launch");
    count_launches(1);
    return RADON_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace of the power iteration: z, w (FP32 images), t (FP32 sinogram), the packed workspaces of
// the forward and the adjoint for one FP32 image, the dot partials and four FP32 scalars.
struct PowerLayout {
    size_t z, w, t, fws, fws_bytes, bws, bws_bytes, partial, scal, total;
};

PowerLayout power_layout(const radon_geometry* g) {
    PowerLayout L;
    const size_t img = (size_t)g->n * g->n * 4, sino = (size_t)g->V * g->D * 4;
    L.z = 0;
    L.w = align_up(L.z + img, 256);
    L.t = align_up(L.w + img, 256);
    L.fws = align_up(L.t + sino, 256);
    L.fws_bytes = std::max(packed_image_bytes(g->n, 1, RADON_F32), single_forward_workspace_bytes(g, RADON_F32));
    L.bws = align_up(L.fws + L.fws_bytes, 256);
    L.bws_bytes = packed_sino_bytes(g->V, g->D, 1, backward_packed_images_per_cta(g, 1, RADON_F32, nullptr), RADON_F32);
    L.partial = align_up(L.bws + L.bws_bytes, 256);
    L.scal = align_up(L.partial + kDotBlocks * sizeof(double), 256);
    L.total = align_up(L.scal + 4 * sizeof(float), 256);
    return L;
}

}  // namespace

}  // namespace radon

using namespace radon;

extern "C" RADON_API size_t radon_dot_workspace_size(void) { return (size_t)kDotBlocks * sizeof(double); }

extern "C" RADON_API radon_status radon_dot(const void* a, const void* b, radon_dtype dtype, int64_t count, float scale,
                                            float* result, int accumulate, void* workspace, size_t workspace_bytes,
                                            void* stream) {
    if (!valid_dtype(dtype)) return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    if (count < 0) return fail(RADON_ERR_INVALID_ARG, "count must be >= 0");
    if (result == nullptr || ((uintptr_t)result & 3) != 0)
        return fail(RADON_ERR_INVALID_ARG, "result must be a 4-byte aligned device pointer");
    if (count > 0 && (a == nullptr || b == nullptr)) return fail(RADON_ERR_INVALID_ARG, "NULL operand with count > 0");
    const size_t es = esize(dtype);
    if (count > 0 && (((uintptr_t)a % es) != 0 || ((uintptr_t)b % es) != 0))
        return fail(RADON_ERR_INVALID_ARG, "operands must be aligned to their element size");
    if (workspace == nullptr || ((uintptr_t)workspace & 7) != 0 || workspace_bytes < radon_dot_workspace_size())
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 8-byte aligned and hold radon_dot_workspace_size() bytes");
    if (!std::isfinite(scale)) return fail(RADON_ERR_INVALID_ARG, "scale must be finite");
    return dot_launch(a, b, dtype, count, scale, result, accumulate, (double*)workspace, (cudaStream_t)stream);
}

extern "C" RADON_API radon_status radon_axpby(const void* x, radon_dtype x_dtype, void* y, radon_dtype y_dtype,
                                              int64_t count, float alpha, const float* alpha_dev, float beta,
                                              void* stream) {
    if (!valid_dtype(x_dtype) || !valid_dtype(y_dtype))
        return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    if (count < 0) return fail(RADON_ERR_INVALID_ARG, "count must be >= 0");
    if (count > 0 && (x == nullptr || y == nullptr)) return fail(RADON_ERR_INVALID_ARG, "NULL operand with count > 0");
    if (count > 0 && (((uintptr_t)x % esize(x_dtype)) != 0 || ((uintptr_t)y % esize(y_dtype)) != 0))
        return fail(RADON_ERR_INVALID_ARG, "operands must be aligned to their element size");
    if (alpha_dev != nullptr && ((uintptr_t)alpha_dev & 3) != 0)
        return fail(RADON_ERR_INVALID_ARG, "alpha_dev must be 4-byte aligned");
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(RADON_ERR_INVALID_ARG, "alpha and beta must be finite");
    return axpby_launch(x, x_dtype, y, y_dtype, count, alpha, alpha_dev, beta, (cudaStream_t)stream);
}

extern "C" RADON_API size_t radon_power_iteration_workspace_size(const radon_geometry* g) {
    if (g == nullptr || g->magic != kGeometryMagic) return 0;
    return power_layout(g).total;
}

extern "C" RADON_API radon_status radon_power_iteration(const radon_geometry* g, const float* v0, int iterations,
                                                        float* lambda_out, float* alpha_out, void* workspace,
                                                        size_t workspace_bytes, void* stream) {
    if (g == nullptr || g->magic != kGeometryMagic)
        return fail(RADON_ERR_INVALID_ARG, "geometry handle is not a live geometry");
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (v0 == nullptr || ((uintptr_t)v0 & 3) != 0) return fail(RADON_ERR_INVALID_ARG, "v0 must be an aligned device pointer");
    if (lambda_out == nullptr || ((uintptr_t)lambda_out & 3) != 0)
        return fail(RADON_ERR_INVALID_ARG, "lambda_out must be an aligned device pointer");
    if (alpha_out != nullptr && ((uintptr_t)alpha_out & 3) != 0)
        return fail(RADON_ERR_INVALID_ARG, "alpha_out must be 4-byte aligned");
    if (iterations < 1) return fail(RADON_ERR_INVALID_ARG, "iterations must be >= 1");
    const PowerLayout L = power_layout(g);
    if (workspace == nullptr || ((uintptr_t)workspace & 15) != 0 || workspace_bytes < L.total)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned and hold "
                                           "radon_power_iteration_workspace_size() bytes");
    radon_status st = check_device(g);
    if (st != RADON_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)workspace;
    float* z = (float*)(ws + L.z);
    float* w = (float*)(ws + L.w);
    float* t = (float*)(ws + L.t);
    double* partial = (double*)(ws + L.partial);
    float* scal = (float*)(ws + L.scal);   // [0] |.|^2, [1] 1 / |.|
    const long long npix = (long long)g->n * g->n;
    // z = v0 / |v0|
    st = dot_launch(v0, v0, RADON_F32, npix, 1.0f, &scal[0], 0, partial, s);
    if (st != RADON_OK) return st;
    rsqrt_kernel<<<1, 32, 0, s>>>(&scal[0], &scal[1]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "power iteration launch");
    count_launches(1);
    st = axpby_launch(v0, RADON_F32, z, RADON_F32, npix, 1.0f, &scal[1], 0.0f, s);
    if (st != RADON_OK) return st;
    for (int it = 0; it < iterations; ++it) {
        st = project(g, z, t, RADON_F32, 1, nullptr, stream, true, ws + L.fws, L.fws_bytes, nullptr);
        if (st != RADON_OK) return st;
        st = project(g, t, w, RADON_F32, 1, nullptr, stream, false, ws + L.bws, L.bws_bytes, nullptr);
        if (st != RADON_OK) return st;
        st = dot_launch(z, w, RADON_F32, npix, 1.0f, lambda_out, 0, partial, s);   // Rayleigh quotient, |z| = 1
        if (st != RADON_OK) return st;
        st = dot_launch(w, w, RADON_F32, npix, 1.0f, &scal[0], 0, partial, s);
        if (st != RADON_OK) return st;
        rsqrt_kernel<<<1, 32, 0, s>>>(&scal[0], &scal[1]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "power iteration launch");
        count_launches(1);
        st = axpby_launch(w, RADON_F32, z, RADON_F32, npix, 1.0f, &scal[1], 0.0f, s);
        if (st != RADON_OK) return st;
    }
    if (alpha_out != nullptr) {
        reciprocal_kernel<<<1, 32, 0, s>>>(lambda_out, alpha_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "power iteration launch");
        count_launches(1);
    }
    return RADON_OK;
}

extern "C" RADON_API size_t radon_dot_batched_workspace_size(int batch) {
    if (batch < 1) return 0;
    return (size_t)batch * dot_blocks(batch) * sizeof(double);
}

extern "C" RADON_API radon_status radon_dot_batched(const void* a, const void* b, radon_dtype dtype, int batch,
                                                    int64_t count, float scale, float* result, int accumulate,
                                                    void* workspace, size_t workspace_bytes, void* stream) {
    if (!valid_dtype(dtype)) return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    if (batch < 0 || count < 0) return fail(RADON_ERR_INVALID_ARG, "batch and count must be >= 0");
    if (batch > 65535) return fail(RADON_ERR_INVALID_ARG, "batch above 65535");
    if (batch == 0) return RADON_OK;
    if (result == nullptr || ((uintptr_t)result & 3) != 0)
        return fail(RADON_ERR_INVALID_ARG, "result must be a 4-byte aligned device pointer");
    if (count > 0 && (a == nullptr || b == nullptr)) return fail(RADON_ERR_INVALID_ARG, "NULL operand with count > 0");
    const size_t es = esize(dtype);
    if (count > 0 && (((uintptr_t)a % es) != 0 || ((uintptr_t)b % es) != 0))
        return fail(RADON_ERR_INVALID_ARG, "operands must be aligned to their element size");
    if (workspace == nullptr || ((uintptr_t)workspace & 7) != 0 ||
        workspace_bytes < radon_dot_batched_workspace_size(batch))
        return fail(RADON_ERR_INVALID_ARG,
                    "workspace must be 8-byte aligned and hold radon_dot_batched_workspace_size(batch) bytes");
    if (!std::isfinite(scale)) return fail(RADON_ERR_INVALID_ARG, "scale must be finite");
    return dot_launch(a, b, dtype, batch, count, scale, result, accumulate, (double*)workspace, (cudaStream_t)stream);
}

extern "C" RADON_API radon_status radon_axpby_batched(const void* x, radon_dtype x_dtype, void* y, radon_dtype y_dtype,
                                                      int batch, int64_t count, float alpha, const float* alpha_dev,
                                                      float beta, const float* beta_dev, void* stream) {
    if (!valid_dtype(x_dtype) || !valid_dtype(y_dtype))
        return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    if (batch < 0 || count < 0) return fail(RADON_ERR_INVALID_ARG, "batch and count must be >= 0");
    if ((long long)batch * count > 0 && (x == nullptr || y == nullptr))
        return fail(RADON_ERR_INVALID_ARG, "NULL operand with elements to update");
    if ((long long)batch * count > 0 &&
        (((uintptr_t)x % esize(x_dtype)) != 0 || ((uintptr_t)y % esize(y_dtype)) != 0))
        return fail(RADON_ERR_INVALID_ARG, "operands must be aligned to their element size");
    if ((alpha_dev != nullptr && ((uintptr_t)alpha_dev & 3) != 0) || (beta_dev != nullptr && ((uintptr_t)beta_dev & 3) != 0))
        return fail(RADON_ERR_INVALID_ARG, "per-item scalars must be 4-byte aligned");
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(RADON_ERR_INVALID_ARG, "alpha and beta must be finite");
    return axpby_launch(x, x_dtype, y, y_dtype, batch, count, alpha, alpha_dev, beta, beta_dev, (cudaStream_t)stream);
}

extern "C" RADON_API radon_status radon_safe_divide(const float* num, const float* den, float* out, int batch,
                                                    void* stream) {
    if (batch < 0) return fail(RADON_ERR_INVALID_ARG, "batch must be >= 0");
    if (batch == 0) return RADON_OK;
    if (num == nullptr || den == nullptr || out == nullptr || (((uintptr_t)num | (uintptr_t)den | (uintptr_t)out) & 3))
        return fail(RADON_ERR_INVALID_ARG, "num, den and out must be 4-byte aligned device pointers");
    return divide_launch(num, den, out, batch, (cudaStream_t)stream);
}

namespace radon {
namespace {

// Workspace of CGNE: r, q (sinograms), s, p (images), FP32; the projections' packed workspaces; the
// batched-dot partials; five per-item scalars (gamma, |q|^2, alpha, gamma', beta).
struct CgneLayout {
    size_t r, q, s, p, fws, fws_bytes, bws, bws_bytes, partial, scal, total;
};

CgneLayout cgne_layout(const radon_geometry* g, int batch) {
    CgneLayout L;
    const size_t sino = (size_t)batch * g->V * g->D * 4, img = (size_t)batch * g->n * g->n * 4;
    L.r = 0;
    L.q = align_up(L.r + sino, 256);
    L.s = align_up(L.q + sino, 256);
    L.p = align_up(L.s + img, 256);
    L.fws = align_up(L.p + img, 256);
    L.fws_bytes = batch == 1 ? std::max(packed_image_bytes(g->n, 1, RADON_F32), single_forward_workspace_bytes(g, RADON_F32))
                             : packed_image_bytes(g->n, batch, RADON_F32);
    L.bws = align_up(L.fws + L.fws_bytes, 256);
    L.bws_bytes = packed_sino_bytes(g->V, g->D, batch, backward_packed_images_per_cta(g, batch, RADON_F32, nullptr), RADON_F32);
    L.partial = align_up(L.bws + L.bws_bytes, 256);
    L.scal = align_up(L.partial + (size_t)batch * dot_blocks(batch) * sizeof(double), 256);
    L.total = align_up(L.scal + 5 * (size_t)batch * sizeof(float), 256);
    return L;
}

}  // namespace
}  // namespace radon

extern "C" RADON_API size_t radon_cgne_workspace_size(const radon_geometry* g, int batch) {
    if (g == nullptr || g->magic != kGeometryMagic || batch < 1) return 0;
    return cgne_layout(g, batch).total;
}

extern "C" RADON_API radon_status radon_cgne(const radon_geometry* g, const void* y, void* x, radon_dtype dtype,
                                             int batch, int iterations, void* workspace, size_t workspace_bytes,
                                             void* stream) {
    radon_status st = validate_call(g, x, y, dtype, batch);
    if (st != RADON_OK) return st;
    if (dtype != RADON_F32) return fail(RADON_ERR_UNSUPPORTED, "CGNE runs on FP32 storage");
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (iterations < 0) return fail(RADON_ERR_INVALID_ARG, "iterations must be >= 0");
    if (batch > 65535) return fail(RADON_ERR_INVALID_ARG, "batch above 65535");
    if (batch == 0 || iterations == 0) return RADON_OK;
    const CgneLayout L = cgne_layout(g, batch);
    if (workspace == nullptr || ((uintptr_t)workspace & 15) != 0 || workspace_bytes < L.total)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned and hold radon_cgne_workspace_size bytes");
    st = check_device(g);
    if (st != RADON_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)workspace;
    float* r = (float*)(ws + L.r);
    float* q = (float*)(ws + L.q);
    float* sv = (float*)(ws + L.s);
    float* p = (float*)(ws + L.p);
    double* partial = (double*)(ws + L.partial);
    float* gamma = (float*)(ws + L.scal);
    float* qq = gamma + batch;
    float* alpha = qq + batch;
    float* gnew = alpha + batch;
    float* beta = gnew + batch;
    const long long npix = (long long)g->n * g->n, nsino = (long long)g->V * g->D;
    // r = y - A x, s = A^T r, p = s, gamma = |s|^2
    const radon_epilogue resid = {-1.0f, nullptr, 1.0f, y};
    st = project(g, x, r, RADON_F32, batch, nullptr, stream, true, ws + L.fws, L.fws_bytes, &resid);
    if (st == RADON_OK) st = project(g, r, sv, RADON_F32, batch, nullptr, stream, false, ws + L.bws, L.bws_bytes, nullptr);
    if (st == RADON_OK) st = axpby_launch(sv, RADON_F32, p, RADON_F32, batch, npix, 1.0f, nullptr, 0.0f, nullptr, s);
    if (st == RADON_OK) st = dot_launch(sv, sv, RADON_F32, batch, npix, 1.0f, gamma, 0, partial, s);
    for (int it = 0; it < iterations && st == RADON_OK; ++it) {
        st = project(g, p, q, RADON_F32, batch, nullptr, stream, true, ws + L.fws, L.fws_bytes, nullptr);   // q = A p
        if (st == RADON_OK) st = dot_launch(q, q, RADON_F32, batch, nsino, 1.0f, qq, 0, partial, s);
        if (st == RADON_OK) st = divide_launch(gamma, qq, alpha, batch, s);                                   // alpha
        if (st == RADON_OK) st = axpby_launch(p, RADON_F32, x, RADON_F32, batch, npix, 1.0f, alpha, 1.0f, nullptr, s);
        if (st == RADON_OK) st = axpby_launch(q, RADON_F32, r, RADON_F32, batch, nsino, -1.0f, alpha, 1.0f, nullptr, s);
        if (st == RADON_OK)
            st = project(g, r, sv, RADON_F32, batch, nullptr, stream, false, ws + L.bws, L.bws_bytes, nullptr);  // s
        if (st == RADON_OK) st = dot_launch(sv, sv, RADON_F32, batch, npix, 1.0f, gnew, 0, partial, s);
        if (st == RADON_OK) st = divide_launch(gnew, gamma, beta, batch, s);                                  // beta
        if (st == RADON_OK) st = axpby_launch(gnew, RADON_F32, gamma, RADON_F32, 1, batch, 1.0f, nullptr, 0.0f, nullptr, s);
        if (st == RADON_OK) st = axpby_launch(sv, RADON_F32, p, RADON_F32, batch, npix, 1.0f, nullptr, 1.0f, beta, s);
    }
    return st;
}
