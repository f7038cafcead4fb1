// Batch-interleaved packing of an image batch for the packed forward projection.
//
// For image group g (BG consecutive images: 4 FP32 or 8 16-bit), two arrays of 16-byte texels:
//   rows[g][i][j]  = (x[g BG + 0][i][j], ..., x[g BG + BG-1][i][j])
//   cols[g][j][i]  = the same texel, transposed (the compute frame of horizontal-class views)
// Images past the batch end read as zero.  One pass over the batch (HBM-bound); every CTA of the
// forward projection then copies its bands of texels straight into shared memory with TMA.
#include "dtype.cuh"
#include "radon_internal.h"

namespace radon {

namespace {

template <typename T>
__device__ __forceinline__ uint4 pack16(const T* v);

template <>
__device__ __forceinline__ uint4 pack16<float>(const float* v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
}

template <typename T>
__device__ __forceinline__ unsigned bits16(T v) {
    unsigned short u;
    memcpy(&u, &v, 2);
    return u;
}

template <>
__device__ __forceinline__ uint4 pack16<__half>(const __half* v) {
    return make_uint4(bits16(v[0]) | (bits16(v[1]) << 16), bits16(v[2]) | (bits16(v[3]) << 16),
                      bits16(v[4]) | (bits16(v[5]) << 16), bits16(v[6]) | (bits16(v[7]) << 16));
}

template <>
__device__ __forceinline__ uint4 pack16<__nv_bfloat16>(const __nv_bfloat16* v) {
    return make_uint4(bits16(v[0]) | (bits16(v[1]) << 16), bits16(v[2]) | (bits16(v[3]) << 16),
                      bits16(v[4]) | (bits16(v[5]) << 16), bits16(v[6]) | (bits16(v[7]) << 16));
}

// 32 x 32 pixel tiles; block (32, 8); grid (tiles, tiles, groups).
template <typename T>
__global__ void __launch_bounds__(256) pack_interleaved_kernel(const T* __restrict__ img, uint4* __restrict__ rows,
                                                               uint4* __restrict__ cols, int n, int B) {
    constexpr int BG = 16 / sizeof(T);
    __shared__ uint4 tile[32][33];
    const int g = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const long long npix = (long long)n * n;
    for (int jr = ty; jr < 32; jr += 8) {
        const int r = r0 + jr, c = c0 + tx;
        uint4 t = make_uint4(0, 0, 0, 0);
        if (r < n && c < n) {
            T v[BG];
#pragma unroll
            for (int b = 0; b < BG; ++b) {
                const int im = g * BG + b;
                v[b] = im < B ? img[(long long)im * npix + (long long)r * n + c] : from_f32<T>(0.0f);
            }
            t = pack16<T>(v);
            rows[((long long)g * n + r) * n + c] = t;
        }
        tile[jr][tx] = t;
    }
    __syncthreads();
    for (int jc = ty; jc < 32; jc += 8) {
        const int c = c0 + jc, r = r0 + tx;
        if (r < n && c < n) cols[((long long)g * n + c) * n + r] = tile[tx][jc];
    }
}

// Sinogram batch -> rows of bg images per detector, [group][view][det][row] in the storage type, row =
// bg elements (16-bit) or bg + 4 (FP32: four padding words, never read, keep the row pitch an odd
// number of 16-byte units).  One thread per row; consecutive threads walk detectors, so the reads of
// each image coalesce and the rows are written contiguously.
template <typename T>
__global__ void __launch_bounds__(256) pack_sino_kernel(const T* __restrict__ y, unsigned char* __restrict__ out,
                                                        int V, int D, int B, int bg, int row_bytes, long long rows) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows) return;
    const int d = (int)(idx % D);
    const long long rest = idx / D;
    const int v = (int)(rest % V);
    const int g = (int)(rest / V);
    constexpr int PER = 16 / sizeof(T);   // elements per 16-byte store
    uint4* dst = reinterpret_cast<uint4*>(out + idx * row_bytes);
    for (int c = 0; c < bg / PER; ++c) {
        T v16[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int b = g * bg + c * PER + u;
            v16[u] = b < B ? y[((long long)b * V + v) * D + d] : from_f32<T>(0.0f);
        }
        dst[c] = pack16<T>(v16);
    }
}

}  // namespace

int packed_sino_row_bytes(int bg, radon_dtype dt) { return dt == RADON_F32 ? (bg + 4) * 4 : bg * 2; }

size_t packed_sino_bytes(int V, int D, int batch, int bg, radon_dtype dt) {
    const long long groups = (batch + bg - 1) / bg;
    return (size_t)(groups * (long long)V * D * packed_sino_row_bytes(bg, dt));
}

cudaError_t launch_pack_sino(const void* sino, void* workspace, int V, int D, int batch, int bg, radon_dtype dt,
                             cudaStream_t s) {
    const long long groups = (batch + bg - 1) / bg;
    const long long rows = groups * (long long)V * D;
    if (rows == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((rows + 255) / 256);
    unsigned char* out = reinterpret_cast<unsigned char*>(workspace);
    const int rb = packed_sino_row_bytes(bg, dt);
    switch (dt) {
        case RADON_F16:
            pack_sino_kernel<__half><<<blocks, 256, 0, s>>>((const __half*)sino, out, V, D, batch, bg, rb, rows);
            break;
        case RADON_BF16:
            pack_sino_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)sino, out, V, D, batch, bg,
                                                                   rb, rows);
            break;
        default:
            pack_sino_kernel<float><<<blocks, 256, 0, s>>>((const float*)sino, out, V, D, batch, bg, rb, rows);
            break;
    }
    return cudaGetLastError();
}

size_t packed_image_bytes(int n, int batch, radon_dtype dt) {
    const int bg = dt == RADON_F32 ? 4 : 8;
    const long long groups = (batch + bg - 1) / bg;
    return (size_t)(2 * groups * (long long)n * n * 16);
}

cudaError_t launch_pack_images(const void* img, void* workspace, int n, int batch, radon_dtype dt, cudaStream_t s) {
    const int bg = dt == RADON_F32 ? 4 : 8;
    const int groups = (batch + bg - 1) / bg;
    if (groups == 0) return cudaSuccess;
    uint4* rows = reinterpret_cast<uint4*>(workspace);
    uint4* cols = rows + (size_t)groups * n * n;
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)groups);
    const dim3 block(32, 8);
    switch (dt) {
        case RADON_F16:
            pack_interleaved_kernel<__half><<<grid, block, 0, s>>>((const __half*)img, rows, cols, n, batch);
            break;
        case RADON_BF16:
            pack_interleaved_kernel<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16*)img, rows, cols, n,
                                                                          batch);
            break;
        default:
            pack_interleaved_kernel<float><<<grid, block, 0, s>>>((const float*)img, rows, cols, n, batch);
            break;
    }
    return cudaGetLastError();
}

}  // namespace radon
