// Sinogram filtering for filtered backprojection (Section 3.1.3).
//
// The Fourier filter of Kak & Slaney (Chapter 3, Eq. 61) is the DFT of the band-limited ramp kernel
// h(0) = 1/4, h(m) = -1 / (pi^2 m^2) for odd m, 0 for even m != 0, zero-padded to P >= 2D - 1, times
// a window of the normalised frequency.  Applied to a zero-padded projection it is a circular
// convolution that, thanks to the padding, equals the linear convolution of the D bins with the
// kernel k = IDFT(filter) at offsets -(D-1) .. D-1.  The taps (pi / V) k are computed here once per
// geometry in FP64 (a radix-2 FFT for the windowed filters; Ram-Lak's taps are the closed form) and
// the kernel sums the linear convolution directly in FP32 -- a few dozen microseconds for a whole
// sinogram batch, with no FFT on the device.  Each tap is stored as an FP32 pair hi + lo: a high-pass
// filter cancels terms up to ~150 times the result, and one FP32 rounding per tap (fixed, so it
// does not average out) would leave a systematic 1e-5-level error; the pair removes it.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "dtype.cuh"
#include "radon_internal.h"

namespace radon {

namespace {

constexpr int kFilterKinds = 5;
constexpr int kFilterThreads = 256;
constexpr int kFilterOut = 4;    // consecutive outputs per thread

using cd = std::complex<double>;

// In-place radix-2 FFT of length a.size() (a power of two); inverse without the 1/P factor.
void fft(std::vector<cd>& a, bool inverse) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = 2.0 * M_PI / (double)len * (inverse ? 1.0 : -1.0);
        const cd wl(std::cos(ang), std::sin(ang));
        for (size_t i = 0; i < n; i += len) {
            cd w(1.0, 0.0);
            for (size_t k = 0; k < len / 2; ++k) {
                const cd u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
                w *= wl;
            }
        }
    }
}

double ramp(long long m) {
    if (m == 0) return 0.25;
    if ((m & 1) == 0) return 0.0;
    return -1.0 / (M_PI * M_PI * (double)m * (double)m);
}

double window(int kind, double f) {
    switch (kind) {
        case RADON_FILTER_SHEPP_LOGAN: return f == 0.0 ? 1.0 : std::sin(M_PI * f) / (M_PI * f);
        case RADON_FILTER_COSINE: return std::cos(M_PI * f);
        case RADON_FILTER_HAMMING: return 0.54 + 0.46 * std::cos(2.0 * M_PI * f);
        case RADON_FILTER_HANN: return 0.5 + 0.5 * std::cos(2.0 * M_PI * f);
        default: return 1.0;
    }
}

// One row: out[d] = sum_{d'} y[d'] taps[d - d' + D - 1], kFilterOut outputs per thread; each tap is
// a (hi, lo) pair summed into two accumulators.
template <typename T>
__global__ void __launch_bounds__(kFilterThreads) filter_rows_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                     const float2* __restrict__ taps, int D) {
    extern __shared__ float fsm[];
    const int Dp = (D + kFilterOut - 1) / kFilterOut * kFilterOut;   // bins padded to whole output groups
    float* y = fsm;                                           // [Dp], zero past D
    float2* t = reinterpret_cast<float2*>(fsm + Dp + (Dp & 1));   // taps at offset +kFilterOut
    const long long row = blockIdx.x;
    const T* src = in + row * D;
    for (int d = threadIdx.x; d < Dp; d += blockDim.x) y[d] = d < D ? to_f32(src[d]) : 0.0f;
    const int nt = 2 * Dp + 2 * kFilterOut;
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        const int m = j - kFilterOut;    // tap index relative to taps[0]
        t[j] = (m >= 0 && m < 2 * D - 1) ? taps[m] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    T* dst = out + row * D;
    for (int d0 = threadIdx.x * kFilterOut; d0 < D; d0 += blockDim.x * kFilterOut) {
        float hi[kFilterOut], lo[kFilterOut];
#pragma unroll
        for (int o = 0; o < kFilterOut; ++o) hi[o] = lo[o] = 0.0f;
        // tap of output d0 + o and input d' sits at t[d0 + o - d' + D - 1 + kFilterOut]; the taps
        // of consecutive inputs slide by one, so a register window takes one new tap per input
        const float2* tb = t + d0 + D - 1 + kFilterOut;
        float2 w[kFilterOut];
#pragma unroll
        for (int o = 0; o < kFilterOut; ++o) w[o] = tb[o];
        for (int q = 0; q < Dp; q += kFilterOut) {
#pragma unroll
            for (int u = 0; u < kFilterOut; ++u) {
                const float yv = y[q + u];
#pragma unroll
                for (int o = 0; o < kFilterOut; ++o) {
                    hi[o] = fmaf(yv, w[o].x, hi[o]);
                    lo[o] = fmaf(yv, w[o].y, lo[o]);
                }
#pragma unroll
                for (int o = kFilterOut - 1; o > 0; --o) w[o] = w[o - 1];
                w[0] = tb[-(q + u + 1)];
            }
        }
#pragma unroll
        for (int o = 0; o < kFilterOut; ++o)
            if (d0 + o < D) dst[d0 + o] = from_f32<T>(hi[o] + lo[o]);
    }
}

size_t filter_smem(int D) {
    const int Dp = (D + kFilterOut - 1) / kFilterOut * kFilterOut;
    return (size_t)(Dp + (Dp & 1)) * sizeof(float) + (size_t)(2 * Dp + 2 * kFilterOut) * sizeof(float2);
}

}  // namespace

radon_status upload_filter_taps(radon_geometry* g) {
    const int D = g->D;
    const long long n_taps = 2LL * D - 1;
    size_t P = 2;   // at least one positive and the Nyquist frequency (D = 1 still filters)
    while ((long long)P < n_taps) P <<= 1;
    std::vector<double> kpad(P);
    for (size_t m = 0; m < P; ++m) kpad[m] = ramp(m <= P / 2 ? (long long)m : (long long)m - (long long)P);
    std::vector<cd> H(P);
    for (size_t m = 0; m < P; ++m) H[m] = cd(kpad[m], 0.0);
    fft(H, false);
    std::vector<float2> taps((size_t)kFilterKinds * n_taps);
    const double scale = M_PI / (double)g->V;
    for (int kind = 0; kind < kFilterKinds; ++kind) {
        std::vector<double> k(P);
        if (kind == RADON_FILTER_RAM_LAK) {
            k = kpad;   // IDFT(DFT(kernel)) is the kernel itself
        } else {
            std::vector<cd> F(P);
            for (size_t m = 0; m < P; ++m) {
                const double f = (m < P / 2 ? (double)m : (double)m - (double)P) / (double)P;   // fftfreq
                F[m] = cd(H[m].real() * window(kind, f), 0.0);
            }
            fft(F, true);
            for (size_t m = 0; m < P; ++m) k[m] = F[m].real() / (double)P;
        }
        for (long long j = 0; j < n_taps; ++j) {
            const long long m = j - (D - 1);
            const double v = scale * k[(size_t)((m % (long long)P + (long long)P) % (long long)P)];
            const float vh = (float)v;
            taps[(size_t)kind * n_taps + j] = make_float2(vh, (float)(v - (double)vh));
        }
    }
    cudaError_t e = cudaMalloc(&g->d_filter_taps, taps.size() * sizeof(float2));
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(RADON_ERR_OOM, "device allocation of filter taps failed")
                                              : cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(g->d_filter_taps, taps.data(), taps.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy filter taps");
    return RADON_OK;
}

}  // namespace radon

using namespace radon;

extern "C" RADON_API radon_status radon_filter_sinogram(const radon_geometry* g, const void* sino, void* out,
                                                        radon_dtype dtype, int batch, radon_filter filter,
                                                        void* stream) {
    radon_status st = validate_call(g, sino, out, dtype, batch);
    if (st != RADON_OK) return st;
    if ((int)filter < 0 || (int)filter >= kFilterKinds) return fail(RADON_ERR_INVALID_ARG, "unknown filter");
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    const size_t es = dtype == RADON_F32 ? 4 : 2;
    const long long rows = (long long)batch * g->V;
    const size_t bytes = (size_t)rows * g->D * es;
    const uintptr_t a = (uintptr_t)sino, b = (uintptr_t)out;
    if (batch > 0 && a < b + bytes && b < a + bytes) return fail(RADON_ERR_INVALID_ARG, "out overlaps sino");
    if (batch == 0) return RADON_OK;
    const size_t smem = filter_smem(g->D);
    if (smem > 227 * 1024) return fail(RADON_ERR_UNSUPPORTED, "det_count too large for the filter kernel");
    if (rows > 0x7fffffffLL) return fail(RADON_ERR_UNSUPPORTED, "too many sinogram rows");
    st = check_device(g);
    if (st != RADON_OK) return st;
    const float2* taps = g->d_filter_taps + (size_t)filter * (2LL * g->D - 1);
    cudaStream_t s = (cudaStream_t)stream;
    // one thread per kFilterOut outputs of the row, in whole warps, at most kFilterThreads
    const int groups = (g->D + kFilterOut - 1) / kFilterOut;
    const int threads = std::min(kFilterThreads, (groups + 31) / 32 * 32);
    cudaError_t e;
    switch (dtype) {
        case RADON_F16:
            e = cudaFuncSetAttribute(filter_rows_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                filter_rows_kernel<__half><<<(unsigned)rows, threads, smem, s>>>((const __half*)sino, (__half*)out,
                                                                                       taps, g->D);
            break;
        case RADON_BF16:
            e = cudaFuncSetAttribute(filter_rows_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                filter_rows_kernel<__nv_bfloat16><<<(unsigned)rows, threads, smem, s>>>(
                    (const __nv_bfloat16*)sino, (__nv_bfloat16*)out, taps, g->D);
            break;
        default:
            e = cudaFuncSetAttribute(filter_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                filter_rows_kernel<float><<<(unsigned)rows, threads, smem, s>>>((const float*)sino, (float*)out,
                                                                                      taps, g->D);
            break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    count_launches(1);
    return RADON_OK;
}
