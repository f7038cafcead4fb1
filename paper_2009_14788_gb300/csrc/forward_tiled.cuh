// Tiled forward projection: y[b][v][d] = h * sum_k bilinear(x_b, sample k of ray (v, d)).
//
// One CTA owns the rays of G views x Dt detectors (one ray per consumer thread, G * Dt = 256) for
// BG images and streams the image through shared memory in slabs of R rows of its "compute frame":
// image rows for views whose rays run mostly along y, image columns (a transposed frame) for the
// others, so every ray advances monotonically through the slabs.
//
// Warp-specialised pipeline, no CTA-wide barrier in the slab loop:
//   * the producer warp bounds the working band of slab s+1 (the columns crossed by the CTA's
//     extreme rays, whose lines enclose every ray of the CTA), issues one 3-D TMA copy of it for all
//     BG images into the staging buffer, waits for it (bounded), waits until the consumers have
//     released the compute buffer it will fill, and repacks the band into 16-byte texels
//     [row][col][image] (BG = 4 FP32 or 8 16-bit values; transposed for the horizontal class);
//   * the 8 consumer warps wait for a full buffer, march their rays through the slab -- one
//     position / floor / weight computation per sample serves all BG images, four 16-byte shared
//     loads fetch the 2x2 texels of every image -- and release the buffer.
// Each ray re-bases its next sample on the band origin from the split-precision table at every
// slab.  All waits are bounded; on expiry the kernel records RADON_ERR_TIMEOUT and unwinds.
// The packed variant (the image batch already packed into texels) copies each band with one 4-D TMA
// box straight into its compute buffer, streams only the slabs between the first and the last in
// which one of the CTA's rays has a sample (about half of all slabs on a fan whose detector is wider
// than the image; a CTA whose rays all miss the image streams none), hands its CTAs out centre-out
// along the detector, and may take two texel groups (2 BG images) per CTA: the box then lands both
// groups' bands as planes of one buffer, and each sample's position and weights serve both.
// Shared memory: header (mbarriers, band origins, abort flag, slab range), staging buffer (repacking
// variant only), compute buffers of (R+2) x wc texels (x NG planes).
#pragma once

#include <type_traits>

#include "device_error.cuh"
#include "dtype.cuh"
#include "epilogue.cuh"
#include "radon_internal.h"
#include "tma.cuh"

namespace radon {

constexpr int kFwdConsumerWarps = 8;
constexpr int kFwdRays = kFwdConsumerWarps * 32;          // rays per CTA
constexpr int kFwdThreads = kFwdRays + 32;                // + one producer warp

struct FwdTiledArgs {
    const RayT* rays;
    const int* nks;
    const Int2* groups;   // (first view, count | class << 16) for this G
    void* sino;
    int n, V, D, B;
    float h;
    int G, Dt;            // views and detectors per CTA (G * Dt * lanes per ray == kFwdRays)
    int pair_views;       // 1: each 8-lane load phase holds two views x four detectors
    int n_dr;             // detector ranges
    int R;                // slab rows (even)
    int n_slabs;
    int wbox;             // band columns (TMA extent along the compute-frame x)
    int wc;               // compute-buffer row pitch in texels
    int rbox_h;           // horizontal class: TMA extent along compute rows (>= R + 2 + align - 2)
    int align;            // elements per 16 B
    int stage_bytes;
    int* err;
    uint32_t spin_limit;
    Epilogue ep;
    int stages;           // compute buffers in the ring (packed: 2..4; repacking: 2)
    int vec_store;        // 1: D even and the sinogram aligned to two elements (paired stores)
};

// Two consecutive outputs as one 4-byte (16-bit storage) or 8-byte (FP32) store; `p` is aligned to
// two elements.
template <typename T>
__device__ __forceinline__ void store_pair(T* p, float lo, float hi);
template <>
__device__ __forceinline__ void store_pair<float>(float* p, float lo, float hi) {
    *reinterpret_cast<float2*>(p) = make_float2(lo, hi);
}
template <>
__device__ __forceinline__ void store_pair<__half>(__half* p, float lo, float hi) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(lo, hi);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, float lo, float hi) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
}

constexpr int kFwdMaxStages = 4;

__host__ __device__ inline size_t fwd_comp_bytes(int R, int wc) { return (size_t)(R + 2) * wc * 16; }

// Packed variant: each ring buffer holds NG image groups' bands, one plane of (R + 2) x wbox texels each.
__host__ __device__ inline size_t fwd_packed_smem_bytes(int R, int wbox, int stages, int NG = 1) {
    return 128 + 128 + (size_t)stages * ((NG * fwd_comp_bytes(R, wbox) + 127) / 128 * 128);
}

__host__ __device__ inline size_t fwd_smem_bytes(int stage_bytes, int R, int wc) {
    return 128 + 128 + (size_t)(stage_bytes + 127) / 128 * 128 + 2 * ((fwd_comp_bytes(R, wc) + 127) / 128 * 128);
}

// 16-byte texel: BG values of one pixel (element b = image b), accumulated with weight w into Acc.
// Arithmetic modes (both accumulate in FP32):
//   kMathScalar  FP32 weights, texel values converted to FP32, one FP32 FMA per image (the default
//                for every storage type: the paper's single-precision arithmetic);
//   kMathF16W    FP16 storage only, opt-in: the weight is rounded once to FP16 and each product of two
//                FP16 values is formed exactly and added in FP32 by one mixed-precision FMA
//                (fma.rn.f32.f16), so nothing converts the texel values; the weight's rounding
//                (relative <= 2^-12) is the only change.
constexpr int kMathScalar = 0;
constexpr int kMathF16W = 1;

template <int BG>
struct AccF {
    float v[BG];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int b = 0; b < BG; ++b) v[b] = 0.0f;
    }
    __device__ __forceinline__ float get(int b) const { return v[b]; }
};

template <typename T, int MODE = kMathScalar>
struct Texel;

template <>
struct Texel<float, kMathScalar> {
    static constexpr int BG = 4;
    using W = float;
    using Acc = AccF<BG>;
    __device__ __forceinline__ static W weight(float w) { return w; }
    __device__ __forceinline__ static void fma(Acc& acc, W w, const uint4& t) {
        acc.v[0] = fmaf(w, __uint_as_float(t.x), acc.v[0]);
        acc.v[1] = fmaf(w, __uint_as_float(t.y), acc.v[1]);
        acc.v[2] = fmaf(w, __uint_as_float(t.z), acc.v[2]);
        acc.v[3] = fmaf(w, __uint_as_float(t.w), acc.v[3]);
    }
};

template <>
struct Texel<__half, kMathScalar> {
    static constexpr int BG = 8;
    using W = float;
    using Acc = AccF<BG>;
    __device__ __forceinline__ static W weight(float w) { return w; }
    __device__ __forceinline__ static void fma2(float* acc, W w, unsigned u) {
        __half2 h2;
        memcpy(&h2, &u, 4);
        const float2 f = __half22float2(h2);
        acc[0] = fmaf(w, f.x, acc[0]);
        acc[1] = fmaf(w, f.y, acc[1]);
    }
    __device__ __forceinline__ static void fma(Acc& acc, W w, const uint4& t) {
        fma2(acc.v, w, t.x);
        fma2(acc.v + 2, w, t.y);
        fma2(acc.v + 4, w, t.z);
        fma2(acc.v + 6, w, t.w);
    }
};

__device__ __forceinline__ float mixed_fma_f16(unsigned short w, unsigned short q, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(w), "h"(q), "f"(c));
    return d;
}

template <>
struct Texel<__half, kMathF16W> {
    static constexpr int BG = 8;
    using W = unsigned short;
    using Acc = AccF<BG>;
    __device__ __forceinline__ static W weight(float w) { return __half_as_ushort(__float2half_rn(w)); }
    __device__ __forceinline__ static void fma2(float* acc, W w, unsigned u) {
        acc[0] = mixed_fma_f16(w, (unsigned short)(u & 0xffffu), acc[0]);
        acc[1] = mixed_fma_f16(w, (unsigned short)(u >> 16), acc[1]);
    }
    __device__ __forceinline__ static void fma(Acc& acc, W w, const uint4& t) {
        fma2(acc.v, w, t.x);
        fma2(acc.v + 2, w, t.y);
        fma2(acc.v + 4, w, t.z);
        fma2(acc.v + 6, w, t.w);
    }
};

template <>
struct Texel<__nv_bfloat16, kMathScalar> {
    static constexpr int BG = 8;
    using W = float;
    using Acc = AccF<BG>;
    __device__ __forceinline__ static W weight(float w) { return w; }
    __device__ __forceinline__ static void fma2(float* acc, W w, unsigned u) {
        acc[0] = fmaf(w, __uint_as_float(u << 16), acc[0]);
        acc[1] = fmaf(w, __uint_as_float(u & 0xffff0000u), acc[1]);
    }
    __device__ __forceinline__ static void fma(Acc& acc, W w, const uint4& t) {
        fma2(acc.v, w, t.x);
        fma2(acc.v + 2, w, t.y);
        fma2(acc.v + 4, w, t.z);
        fma2(acc.v + 6, w, t.w);
    }
};

struct FwdBand {
    int xc0;    // compute-frame column of buffer column 0
    int xt;     // horizontal class: TMA start along compute rows (aligned); yoff = ylo - xt
    int bad;    // the band exceeded wbox (recorded; rays outside it are skipped)
};

// Producer warp: the lines of the CTA's extreme rays (the first and last detector of each view), one
// per lane in the compute frame, loaded once per CTA: the band of every slab follows from them.
struct FwdEdge {
    float X0, Y0, sl;   // a point of the line and its slope dX / dY
    bool valid, flat;   // flat: the line runs along the slab rows (covers the whole support)
};

__device__ __forceinline__ FwdEdge fwd_edge(const FwdTiledArgs& a, int v0, int cnt, int cls, int d0) {
    const int lane = threadIdx.x & 31;
    FwdEdge e{0.f, 0.f, 0.f, false, false};
    if (lane < 2 * cnt) {
        const int vl = lane >> 1;
        const int d = (lane & 1) ? min(d0 + a.Dt - 1, a.D - 1) : d0;
        const RayT r = a.rays[(long long)(v0 + vl) * a.D + d];
        e.X0 = cls ? (float)r.I0 + r.fy0 : (float)r.J0 + r.fx0;
        e.Y0 = cls ? (float)r.J0 + r.fx0 : (float)r.I0 + r.fy0;
        const float dX = cls ? r.dyh + r.dyl : r.dxh + r.dxl;
        const float dY = cls ? r.dxh + r.dxl : r.dyh + r.dyl;
        e.flat = fabsf(dY) <= 1e-6f * fabsf(dX);
        e.sl = e.flat ? 0.0f : dX / dY;
        e.valid = true;
    }
    return e;
}

// Producer warp: band of slab s (every lane returns it): the columns crossed by the lines of the
// CTA's extreme rays over the slab's buffer rows (+-1 row), clamped to the support, 2 columns of
// margin.  `align_x` aligns the start (TMA needs 16-byte aligned starts along the innermost axis).
__device__ __forceinline__ FwdBand fwd_band(const FwdTiledArgs& a, const FwdEdge& e, int s, int align_x) {
    const int ylo = -4 + s * a.R, yhi = ylo + a.R + 1;   // buffer rows [ylo, yhi]
    float lo = 3.0e38f, hi = -3.0e38f;
    if (e.valid) {
        if (e.flat) {
            lo = -3.0f;
            hi = (float)a.n + 2.0f;
        } else {
            const float xa = fmaf((float)(ylo - 1) - e.Y0, e.sl, e.X0), xb = fmaf((float)(yhi + 1) - e.Y0, e.sl, e.X0);
            lo = fminf(xa, xb);
            hi = fmaxf(xa, xb);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    lo = fmaxf(lo, -3.0f);
    hi = fminf(hi, (float)a.n + 2.0f);
    if (hi < lo) hi = lo;
    const int x_lo = (int)floorf(lo) - 2, x_hi = (int)ceilf(hi) + 2;
    FwdBand band;
    band.xc0 = x_lo - (((x_lo % align_x) + align_x) % align_x);
    band.xt = ylo - (((ylo % a.align) + a.align) % a.align);
    band.bad = (x_hi - band.xc0 + 1 > a.wbox) ? 1 : 0;
    return band;
}

// Producer warp (repacking pipeline): band of slab s and, from lane 0, its TMA copy into staging.
template <typename T>
__device__ FwdBand fwd_issue_slab(const CUtensorMap* map_v, const CUtensorMap* map_h, const FwdTiledArgs& a, int s,
                                  const FwdEdge& edge, int cls, int b0, uint64_t* tma_bar, unsigned char* stage) {
    const int lane = threadIdx.x & 31;
    const int ylo = -4 + s * a.R;
    const FwdBand band = fwd_band(a, edge, s, cls ? 1 : a.align);
    if (lane == 0) {
        fence_proxy_async_shared();
        if (cls == 0) {
            mbar_arrive_expect_tx(tma_bar, (uint32_t)(a.wbox * (a.R + 2) * 16));
            tma_load_3d(stage, map_v, tma_bar, band.xc0, ylo, b0);
        } else {
            mbar_arrive_expect_tx(tma_bar, (uint32_t)(a.rbox_h * a.wbox * 16));
            tma_load_3d(stage, map_h, tma_bar, band.xt, band.xc0, b0);
        }
    }
    __syncwarp();
    return band;
}

// Producer warp: staged band (planar per image) -> compute buffer texels [row][col][image].
// Pairs of adjacent elements are read as one 32-bit (16-bit storage) or 64-bit (FP32) word.
template <typename T>
__device__ void fwd_repack(const FwdTiledArgs& a, int cls, int yoff, const unsigned char* stage, uint4* comp) {
    const int lane = threadIdx.x & 31;
    const int rows = a.R + 2;
    if constexpr (sizeof(T) == 2) {
        const unsigned short* st = reinterpret_cast<const unsigned short*>(stage);
        if (cls == 0) {
            const int half = a.wbox >> 1;
            for (int e = lane; e < rows * half; e += 32) {
                const int r = e / half, c = 2 * (e - (e / half) * half);
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    w[b] = *reinterpret_cast<const unsigned*>(st + ((size_t)b * rows + r) * a.wbox + c);
                comp[r * a.wc + c] = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                                                __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                comp[r * a.wc + c + 1] = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                                                    __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
            }
        } else {
            const int half = rows >> 1;
            for (int e = lane; e < a.wbox * half; e += 32) {
                const int c = e / half, r = 2 * (e - (e / half) * half);
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    w[b] = *reinterpret_cast<const unsigned*>(st + ((size_t)b * a.wbox + c) * a.rbox_h + yoff + r);
                comp[r * a.wc + c] = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                                                __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                comp[(r + 1) * a.wc + c] = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                                                      __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
            }
        }
    } else {
        const float* st = reinterpret_cast<const float*>(stage);
        if (cls == 0) {
            const int half = a.wbox >> 1;
            for (int e = lane; e < rows * half; e += 32) {
                const int r = e / half, c = 2 * (e - (e / half) * half);
                float2 w[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) w[b] = *reinterpret_cast<const float2*>(st + ((size_t)b * rows + r) * a.wbox + c);
                comp[r * a.wc + c] = make_uint4(__float_as_uint(w[0].x), __float_as_uint(w[1].x), __float_as_uint(w[2].x),
                                                __float_as_uint(w[3].x));
                comp[r * a.wc + c + 1] = make_uint4(__float_as_uint(w[0].y), __float_as_uint(w[1].y),
                                                    __float_as_uint(w[2].y), __float_as_uint(w[3].y));
            }
        } else {
            const int half = rows >> 1;
            for (int e = lane; e < a.wbox * half; e += 32) {
                const int c = e / half, r = 2 * (e - (e / half) * half);
                float2 w[4];
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    w[b] = *reinterpret_cast<const float2*>(st + ((size_t)b * a.wbox + c) * a.rbox_h + yoff + r);
                comp[r * a.wc + c] = make_uint4(__float_as_uint(w[0].x), __float_as_uint(w[1].x), __float_as_uint(w[2].x),
                                                __float_as_uint(w[3].x));
                comp[(r + 1) * a.wc + c] = make_uint4(__float_as_uint(w[0].y), __float_as_uint(w[1].y),
                                                      __float_as_uint(w[2].y), __float_as_uint(w[3].y));
            }
        }
    }
}

// Consumer warps: one ray per thread, marched slab by slab through the double-buffered compute
// buffers (texels [row][col][image], row pitch wc), released through `empty` after each slab.  With
// NG = 2 a buffer holds two image groups' texel planes, `plane` bytes apart: one position, floor and
// weight evaluation per sample serves both groups (2 BG images).  With LN = 2 two lanes share each
// ray (rays where bands of 256 detectors per view would not fit a TMA box): lane `sub` takes the
// ray's samples sub, sub + 2, ... of every slab, the two lanes agree on where the slab's samples end,
// and their partial sums meet in one shuffle before the store.
template <typename T, int MODE, int NG = 1, int LN = 1>
__device__ void fwd_consume(const FwdTiledArgs& a, int cls, int v0, int cnt, int d0, int b0, uint64_t* full,
                            uint64_t* empty, const int* band_xc0, const int* band_bad, volatile int* abort_flag,
                            const unsigned char* comp_base, size_t comp_stride, int wc, int* slab_rng,
                            unsigned plane = 0u) {
    using TX = Texel<T, MODE>;
    constexpr int BG = TX::BG;
    const int tid = threadIdx.x;
    // Thread -> (view, detector) of the CTA.  By default consecutive threads take consecutive detectors
    // of one view; with pair_views each 8-lane phase of a 16-byte shared load takes views 2m, 2m + 1 x
    // four consecutive detectors (lanes 2j, 2j + 1 still hold neighbouring detectors of one view).
    int vl, dl;
    const int sub = LN == 2 ? (tid & 1) : 0;
    if (LN == 2) {
        const int r = tid >> 1;
        vl = r / a.Dt;
        dl = r - vl * a.Dt;
    } else if (a.pair_views) {
        const int per = a.Dt >> 2, P = tid >> 3;
        vl = (P / per) * 2 + ((tid >> 2) & 1);
        dl = (P - (P / per) * per) * 4 + (tid & 3);
    } else {
        vl = tid / a.Dt;
        dl = tid - vl * a.Dt;
    }
    const int d = d0 + dl;
    const bool active = vl < cnt && d < a.D;
    int J0 = 0, I0 = 0, nk = 0;
    float fX0 = 0.f, fY0 = 0.f, dXh = 0.f, dYh = 0.f, dXl = 0.f, dYl = 0.f;
    if (active) {
        const long long ridx = (long long)(v0 + vl) * a.D + d;
        const RayT r = a.rays[ridx];
        nk = a.nks[ridx];
        if (cls == 0) {
            J0 = r.J0; I0 = r.I0; fX0 = r.fx0; fY0 = r.fy0; dXh = r.dxh; dYh = r.dyh; dXl = r.dxl; dYl = r.dyl;
        } else {
            J0 = r.I0; I0 = r.J0; fX0 = r.fy0; fY0 = r.fx0; dXh = r.dyh; dYh = r.dxh; dXl = r.dyl; dYl = r.dxl;
        }
    }
    const float dX = dXh + dXl, dY = dYh + dYl;
    // Slabs [s_lo, s_hi] hold the CTA's samples: slab s takes a ray's samples whose compute-frame row
    // Y (= I0 + fY0 + k dY, increasing with k) lies below R (s + 1) - 3, from the first slab on where
    // that holds (the loop below), so sample Y falls in slab floor((Y + 3) / R).  With slab_rng the
    // consumer warps reduce their rays' first and last slabs (a 0.01-row margin absorbs rounding)
    // and the producer streams only that range; slabs outside it would give no ray a sample, so the
    // sums are the same bits.  A CTA none of whose rays meets the image streams nothing.
    int s_lo = 0, s_hi = a.n_slabs - 1;
    if (slab_rng != nullptr) {
        int lo = 0x7fffffff, hi = -1;
        if (nk > 0) {
            const float y0 = (float)I0 + fY0, y1 = fmaf((float)(nk - 1), dY, y0);
            lo = max((int)floorf((fminf(y0, y1) + 2.99f) / (float)a.R), 0);
            hi = min((int)floorf((fmaxf(y0, y1) + 3.01f) / (float)a.R), a.n_slabs - 1);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((tid & 31) == 0) {
            atomicMin(&slab_rng[0], lo);
            atomicMax(&slab_rng[1], hi);
        }
        named_barrier_sync(1, kFwdThreads);   // with the producer warp
        s_lo = slab_rng[0];
        s_hi = slab_rng[1];
    }
    int k = 0;
    typename TX::Acc acc[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) acc[g].zero();

    for (int s = s_lo; s <= s_hi; ++s) {
        const int j = s - s_lo;   // ring position
        const int buf = j % a.stages;
        bool ok = mbar_wait_bounded(&full[buf], (uint32_t)((j / a.stages) & 1), a.spin_limit);
        // two lanes per ray: the warp gives up together, so no lane is left waiting in a shuffle
        if (LN == 2) ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            record_device_error(a.err, RADON_ERR_TIMEOUT);
            return;
        }
        if (*abort_flag) return;
        const int xc0 = band_xc0[buf];
        if (tid == 0 && band_bad[buf]) record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
        const uint4* comp = reinterpret_cast<const uint4*>(comp_base + (size_t)buf * comp_stride);
        if (k < nk) {
            const int ylo = -4 + s * a.R;
            const float kf = (float)k;
            const float qX = kf * dXh, qY = kf * dYh;   // exact products
            const float QX = floorf(qX), QY = floorf(qY);
            const float sX = fmaf(kf, dXl, fX0 + (qX - QX));
            const float sY = fmaf(kf, dYl, fY0 + (qY - QY));
            const int JB = J0 + (int)QX - xc0;   // band-local integer base of sample k
            const int IB = I0 + (int)QY - ylo;
            const float ylim = (s == a.n_slabs - 1) ? 3.0e38f : (float)(a.R + 1 - IB);
            // the ray's next sample may lie in a later slab (rays entering through a side)
            if ((sY - 0.5f) < (ylim - 0.5f)) {
                // every sample of this slab stays inside the band (the extreme rays' lines enclose
                // the CTA's rays); checked per ray so that no access can leave the buffer
                const float xa = (float)JB + sX;
                float steps = (float)(nk - 1 - k);
                if (s != a.n_slabs - 1 && fabsf(dY) > 1e-6f * fabsf(dX)) steps = fminf(steps, (ylim - sY) / dY);
                const float xb = fmaf(steps, dX, xa);
                if (fminf(xa, xb) < 1.0f || fmaxf(xa, xb) > (float)(a.wbox - 2) || IB + sY < 0.5f) {
                    record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
                    k = nk;
                } else {
                    // floors by round-to-nearest of (value - 1/2) through the 1.5 * 2^23 magic
                    // constant; at exact integers either neighbour gives the same bilinear value
                    const float M = 12582912.0f;
                    const unsigned magic = 0x4B400000u;
                    const float sXm = sX - 0.5f, sYm = sY - 0.5f, ylim_m = ylim - 0.5f;
                    const unsigned comp_a = smem_u32(comp);
                    // shared address of texel (row, col) = comp + 16 (row * wc + col): the magic-biased
                    // bit patterns of the floors enter modulo 2^32, so the biases cancel exactly
                    const unsigned wc16 = 16u * (unsigned)wc;
                    const unsigned base16 = comp_a + 16u * ((unsigned)(IB * wc + JB) - magic * (unsigned)(wc + 1));
                    const int kleft = nk - k;
                    int i = sub;
                    float kk = (float)sub;
                    // FP32 texels (4 images per load): a sample one row below the previous one in the
                    // same column takes its upper row from the previous sample's lower row instead of
                    // loading it (same values: same bits; 2-5 % faster in FP32; the 16-bit paths, with
                    // twice the FMAs per load, measured 2-11 % slower and load every texel)
                    constexpr bool kReuseRow = std::is_same<T, float>::value && NG == 1 && LN == 1;
                    unsigned pa = 0x80000000u;   // no texel address of a band lies within a row of it
                    uint4 r10 = make_uint4(0u, 0u, 0u, 0u), r11 = r10;
                    for (; i < kleft; i += LN, kk += (float)LN) {
                        const float fym = fmaf(kk, dY, sYm);
                        if (fym >= ylim_m) break;
                        const float fxm = fmaf(kk, dX, sXm);
                        const float tx = fxm + M, ty = fym + M;
                        const unsigned ad = __float_as_uint(ty) * wc16 + __float_as_uint(tx) * 16u + base16;
                        const float ax = fxm - (tx - M), ay = fym - (ty - M);   // in [-1/2, 1/2]
                        const float wx1 = 0.5f + ax, wx0 = 0.5f - ax, wy1 = 0.5f + ay, wy0 = 0.5f - ay;
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const unsigned adg = ad + (unsigned)g * plane;
                            uint4 q00, q01;
                            if (kReuseRow && adg == pa + wc16) {
                                q00 = r10;
                                q01 = r11;
                            } else {
                                q00 = lds4u(adg);
                                q01 = lds4u(adg + 16u);
                            }
                            const uint4 q10 = lds4u(adg + wc16), q11 = lds4u(adg + wc16 + 16u);
                            if (kReuseRow) {
                                r10 = q10;
                                r11 = q11;
                                pa = adg;
                            }
                            TX::fma(acc[g], TX::weight(wx0 * wy0), q00);
                            TX::fma(acc[g], TX::weight(wx1 * wy0), q01);
                            TX::fma(acc[g], TX::weight(wx0 * wy1), q10);
                            TX::fma(acc[g], TX::weight(wx1 * wy1), q11);
                        }
                    }
                    if (LN == 2) {
                        // the slab's samples end where the first lane stopped (samples advance
                        // monotonically, so the other lane stopped one sample later)
                        const unsigned pair_mask = 3u << (threadIdx.x & 30);
                        i = min(min(i, __shfl_xor_sync(pair_mask, i, 1)), kleft);
                    }
                    k += i;
                }
            }
        }
        mbar_arrive(&empty[buf]);   // this thread's reads of the buffer are done
    }
    // Stores: consecutive lanes hold runs of consecutive detectors of one view (a warp's 32 with one
    // view per load phase, runs of 4 with two), so each image's stores coalesce per run.  With
    // vec_store (D even and the output aligned to two elements, so every even detector's index is
    // even) and the whole warp present, each even lane also takes its odd neighbour's value and writes
    // both as one two-element vector.
    T* out = reinterpret_cast<T*>(a.sino);
    const long long vd = (long long)a.V * a.D;
    const long long o = (long long)(v0 + vl) * a.D + d;
    if (LN == 2) {   // the two lanes' partial sums (every consumer thread is here)
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int b = 0; b < BG; ++b) acc[g].v[b] += __shfl_xor_sync(0xffffffffu, acc[g].v[b], 1);
    }
    const bool pairs = LN == 1 && a.vec_store != 0 && __activemask() == 0xffffffffu;
#pragma unroll
    for (int gb = 0; gb < NG * BG; ++gb) {
        const int b = gb;   // image b0 + b: group b / BG, slot b % BG
        const bool mine = active && sub == 0 && b0 + b < a.B;
        const long long idx = (long long)(b0 + b) * vd + o;
        const float val = mine ? epilogue_value<T>(a.ep, a.h * acc[gb / BG].get(gb % BG), idx) : 0.0f;
        if (pairs) {
            const float nval = __shfl_xor_sync(0xffffffffu, val, 1);
            const bool nmine = __shfl_xor_sync(0xffffffffu, mine ? 1 : 0, 1) != 0;
            const bool even = (threadIdx.x & 1) == 0;
            if (mine && even && nmine)
                store_pair<T>(out + idx, val, nval);
            else if (mine && (even || !nmine))
                out[idx] = from_f32<T>(val);
        } else if (mine) {
            out[idx] = from_f32<T>(val);
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kFwdThreads, 3) forward_tiled_kernel(const __grid_constant__ CUtensorMap map_v,
                                                                      const __grid_constant__ CUtensorMap map_h,
                                                                      const FwdTiledArgs a) {
    constexpr int BG = Texel<T>::BG;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* tma_bar = reinterpret_cast<uint64_t*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + 8);    // [2]
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + 24);  // [2]
    int* band_xc0 = reinterpret_cast<int*>(smem + 40);          // [2]
    int* band_bad = reinterpret_cast<int*>(smem + 48);          // [2]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 56);
    unsigned char* stage = smem + 128;
    const size_t comp_stride = (fwd_comp_bytes(a.R, a.wc) + 127) / 128 * 128;
    unsigned char* comp_base = stage + (a.stage_bytes + 127) / 128 * 128;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int grp_idx = blockIdx.x / a.n_dr, dr = blockIdx.x - (blockIdx.x / a.n_dr) * a.n_dr;
    const Int2 grp = a.groups[grp_idx];
    const int v0 = grp.x, cnt = grp.y & 0xffff, cls = grp.y >> 16;
    const int d0 = dr * a.Dt;
    const int b0 = blockIdx.y * BG;

    if (tid == 0) {
        mbar_init(tma_bar, 1);
        mbar_init(&full[0], 32);
        mbar_init(&full[1], 32);
        mbar_init(&empty[0], kFwdRays);
        mbar_init(&empty[1], kFwdRays);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kFwdConsumerWarps) {
        // ------------------------------------------------------------------ producer warp
        const int lane = tid & 31;
        const FwdEdge edge = fwd_edge(a, v0, cnt, cls, d0);
        FwdBand band = fwd_issue_slab<T>(&map_v, &map_h, a, 0, edge, cls, b0, tma_bar, stage);
        for (int s = 0; s < a.n_slabs; ++s) {
            const int buf = s & 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(tma_bar, (uint32_t)(s & 1), a.spin_limit);
            if (ok && s >= 2 && lane == 0)
                ok = mbar_wait_bounded(&empty[buf], (uint32_t)(((s >> 1) - 1) & 1), a.spin_limit);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) {
                    record_device_error(a.err, RADON_ERR_TIMEOUT);
                    *abort_flag = 1;
                }
                __syncwarp();
                mbar_arrive(&full[buf]);   // wake the consumers so they see the abort
                return;
            }
            const int ylo = -4 + s * a.R;
            fwd_repack<T>(a, cls, ylo - band.xt, stage,
                          reinterpret_cast<uint4*>(comp_base + (size_t)buf * comp_stride));
            if (lane == 0) {
                band_xc0[buf] = band.xc0;
                band_bad[buf] = band.bad;
            }
            __syncwarp();
            mbar_arrive(&full[buf]);        // every lane: its repacked texels are released
            if (s + 1 < a.n_slabs)
                band = fwd_issue_slab<T>(&map_v, &map_h, a, s + 1, edge, cls, b0, tma_bar, stage);
        }
        return;
    }

    fwd_consume<T, MODE>(a, cls, v0, cnt, d0, b0, full, empty, band_xc0, band_bad, abort_flag, comp_base, comp_stride,
                   a.wc, nullptr);
}

// Packed variant: the image batch was packed once into 16-byte texels (rows / cols copies, see
// pack.cu), so the producer warp only bounds each band and copies it with one 4-D TMA load straight
// into the compute buffer it will become (row pitch = band width); no staging, no repack.
template <typename T, int MODE, int NG, int LN>
__global__ void __launch_bounds__(kFwdThreads, 3) forward_packed_kernel(const __grid_constant__ CUtensorMap map_rows,
                                                                       const __grid_constant__ CUtensorMap map_cols,
                                                                       const FwdTiledArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);         // [stages]: TMA completion
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + 32);   // [stages]: consumers released
    int* band_xc0 = reinterpret_cast<int*>(smem + 64);          // [stages]
    int* band_bad = reinterpret_cast<int*>(smem + 80);          // [stages]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 96);
    int* slab_rng = reinterpret_cast<int*>(smem + 104);         // [2]: first, last slab with samples
    const unsigned plane = (unsigned)fwd_comp_bytes(a.R, a.wbox);   // one image group's texels
    const size_t comp_stride = ((size_t)NG * plane + 127) / 128 * 128;
    unsigned char* comp_base = smem + 128;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    // CTAs are handed out in index order, so the detector ranges run centre-out: the ranges whose rays
    // cross the middle of the image (the longest) start first and the short outer ones fill the tail.
    const int n_grp = gridDim.x / a.n_dr;
    const int rank = blockIdx.x / n_grp, grp_idx = blockIdx.x - rank * n_grp;
    const int dr = (rank & 1) ? ((a.n_dr + 1) / 2 + (rank >> 1)) : ((a.n_dr - 1) / 2 - (rank >> 1));
    const Int2 grp = a.groups[grp_idx];
    const int v0 = grp.x, cnt = grp.y & 0xffff, cls = grp.y >> 16;
    const int d0 = dr * a.Dt;
    const int b0 = blockIdx.y * NG * Texel<T>::BG;

    if (tid < a.stages) {
        mbar_init(&full[tid], 1);
        mbar_init(&empty[tid], kFwdRays);
    }
    if (tid == 0) {
        *abort_flag = 0;
        slab_rng[0] = 0x7fffffff;
        slab_rng[1] = -1;
    }
    fence_mbar_init();
    __syncthreads();

    if (warp == kFwdConsumerWarps) {
        const int lane = tid & 31;
        const CUtensorMap* map = cls ? &map_cols : &map_rows;
        const FwdEdge edge = fwd_edge(a, v0, cnt, cls, d0);
        named_barrier_sync(1, kFwdThreads);   // the consumers have reduced the slab range
        const int s_lo = slab_rng[0], s_hi = slab_rng[1];
        for (int s = s_lo; s <= s_hi; ++s) {
            const int j = s - s_lo;
            const int buf = j % a.stages;
            const FwdBand band = fwd_band(a, edge, s, 1);
            bool ok = true;
            if (j >= a.stages && lane == 0)
                ok = mbar_wait_bounded(&empty[buf], (uint32_t)((j / a.stages - 1) & 1), a.spin_limit);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (lane == 0) {
                if (!ok) {
                    record_device_error(a.err, RADON_ERR_TIMEOUT);
                    *abort_flag = 1;
                    mbar_arrive(&full[buf]);   // completes the phase without data: consumers see the abort
                } else {
                    band_xc0[buf] = band.xc0;
                    band_bad[buf] = band.bad;
                    fence_proxy_async_shared();
                    // NG groups' planes in one box (a group past the batch's last reads as zeros)
                    mbar_arrive_expect_tx(&full[buf], (uint32_t)NG * plane);
                    tma_load_4d(comp_base + (size_t)buf * comp_stride, map, &full[buf], 0, band.xc0, -4 + s * a.R,
                                (int)blockIdx.y * NG);
                }
            }
            __syncwarp();
            if (!ok) return;
        }
        return;
    }
    if (NG == 2 && b0 + Texel<T>::BG < a.B)
        fwd_consume<T, MODE, NG, LN>(a, cls, v0, cnt, d0, b0, full, empty, band_xc0, band_bad, abort_flag,
                                     comp_base, comp_stride, a.wbox, slab_rng, plane);
    else   // one group (or a pair whose second group lies past the batch: its plane is never read)
        fwd_consume<T, MODE, 1, LN>(a, cls, v0, cnt, d0, b0, full, empty, band_xc0, band_bad, abort_flag,
                                    comp_base, comp_stride, a.wbox, slab_rng);
}

}  // namespace radon
