// Tiled forward projection: y[b][v][d] = h * sum_k bilinear(x_b, sample k of ray (v, d)).
//
// One CTA owns the rays of G views x Dt detectors (one ray per thread) for BG images and streams
// the image through shared memory in slabs of R rows of its "compute frame": image rows for views
// whose rays run mostly along y, image columns (a transposed frame) for the others, so every ray
// advances monotonically through the slabs.  For each slab:
//   * warp 0 bounds the working band (the columns crossed by the CTA's extreme rays, whose lines
//     enclose every ray of the CTA) and issues one 3-D TMA copy of the band for all BG images
//     into the staging buffer (bounded mbarrier wait);
//   * all threads repack it into the compute buffer as 16-byte texels [row][col][image] (BG = 4
//     FP32 or 8 16-bit values), transposing for the horizontal class;
//   * each ray re-bases its next sample on the band origin from the split-precision table, then
//     steps through the slab: one position, floor and weight computation per sample serves all
//     BG images; four 16-byte shared loads fetch the 2x2 texels of every image.
// The TMA copy of slab s+1 overlaps the compute of slab s.  Shared memory (128 B aligned pieces):
//   header (mbarrier, status, band origin), staging buffer, compute buffer (R+2) x wc texels.
#pragma once

#include "device_error.cuh"
#include "dtype.cuh"
#include "radon_internal.h"
#include "tma.cuh"

namespace radon {

constexpr int kFwdThreads = 256;

struct FwdTiledArgs {
    const RayT* rays;
    const int* nks;
    const Int2* groups;   // (first view, count | class << 16) for this G
    void* sino;
    int n, V, D, B;
    float h;
    int G, Dt;            // views and detectors per CTA (G * Dt == kFwdThreads)
    int n_dr;             // detector ranges
    int R;                // slab rows
    int n_slabs;
    int wbox;             // band columns (TMA extent along the compute-frame x)
    int wc;               // compute-buffer row pitch in texels
    int rbox_h;           // horizontal class: TMA extent along compute rows (>= R + 2 + align - 1)
    int align;            // elements per 16 B
    int stage_bytes;
    int* err;
    uint32_t spin_limit;
};

__host__ __device__ inline size_t fwd_smem_bytes(int stage_bytes, int R, int wc) {
    return 128 + 128 + (size_t)(stage_bytes + 127) / 128 * 128 + (size_t)(R + 2) * wc * 16;
}

// 16-byte texel -> BG floats
template <typename T>
struct TexelCvt;

template <>
struct TexelCvt<float> {
    static constexpr int BG = 4;
    __device__ __forceinline__ static void load(const uint4& t, float* v) {
        v[0] = __uint_as_float(t.x);
        v[1] = __uint_as_float(t.y);
        v[2] = __uint_as_float(t.z);
        v[3] = __uint_as_float(t.w);
    }
};

template <>
struct TexelCvt<__half> {
    static constexpr int BG = 8;
    __device__ __forceinline__ static void load(const uint4& t, float* v) {
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h2;
            memcpy(&h2, &w[i], 4);
            const float2 f = __half22float2(h2);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
};

template <>
struct TexelCvt<__nv_bfloat16> {
    static constexpr int BG = 8;
    __device__ __forceinline__ static void load(const uint4& t, float* v) {
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

// Storage elements -> one 16-byte texel (element b of the texel = image b).
template <typename T>
__device__ __forceinline__ uint4 pack_texel(const T* e);

template <>
__device__ __forceinline__ uint4 pack_texel<float>(const float* e) {
    return make_uint4(__float_as_uint(e[0]), __float_as_uint(e[1]), __float_as_uint(e[2]), __float_as_uint(e[3]));
}

template <typename T>
__device__ __forceinline__ uint4 pack_texel16(const T* e) {
    unsigned short u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) memcpy(&u[i], &e[i], 2);
    return make_uint4((unsigned)u[0] | ((unsigned)u[1] << 16), (unsigned)u[2] | ((unsigned)u[3] << 16),
                      (unsigned)u[4] | ((unsigned)u[5] << 16), (unsigned)u[6] | ((unsigned)u[7] << 16));
}

template <>
__device__ __forceinline__ uint4 pack_texel<__half>(const __half* e) {
    return pack_texel16(e);
}
template <>
__device__ __forceinline__ uint4 pack_texel<__nv_bfloat16>(const __nv_bfloat16* e) {
    return pack_texel16(e);
}

struct FwdBand {
    int xc0;    // compute-frame column of buffer column 0
    int yoff;   // horizontal class: staged row offset of buffer row 0
    int bad;    // the band exceeded wbox (recorded; rays outside it are skipped)
};

// Warp 0: band of slab s and its TMA copy into the staging buffer.
template <typename T>
__device__ void fwd_issue_slab(const CUtensorMap* map_v, const CUtensorMap* map_h, const FwdTiledArgs& a, int s,
                               int v0, int cnt, int cls, int d0, int b0, uint64_t* mbar, FwdBand* band,
                               unsigned char* stage) {
    const int lane = threadIdx.x & 31;
    const int ylo = -3 + s * a.R, yhi = -2 + s * a.R + a.R;
    float lo = 3.0e38f, hi = -3.0e38f;
    if (lane < 2 * cnt) {
        const int vl = lane >> 1;
        const int d = (lane & 1) ? min(d0 + a.Dt - 1, a.D - 1) : d0;
        const RayT r = a.rays[(long long)(v0 + vl) * a.D + d];
        const float X0 = cls ? (float)r.I0 + r.fy0 : (float)r.J0 + r.fx0;
        const float Y0 = cls ? (float)r.J0 + r.fx0 : (float)r.I0 + r.fy0;
        const float dX = cls ? r.dyh + r.dyl : r.dxh + r.dxl;
        const float dY = cls ? r.dxh + r.dxl : r.dyh + r.dyl;
        if (fabsf(dY) <= 1e-6f * fabsf(dX)) {
            lo = -3.0f;
            hi = (float)a.n + 2.0f;
        } else {
            const float sl = dX / dY;
            const float xa = fmaf((float)(ylo - 1) - Y0, sl, X0), xb = fmaf((float)(yhi + 1) - Y0, sl, X0);
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
    const int xc0 = cls ? x_lo : x_lo - (((x_lo % a.align) + a.align) % a.align);
    if (lane == 0) {
        band->xc0 = xc0;
        band->bad = (x_hi - xc0 + 1 > a.wbox) ? 1 : 0;
        uint32_t bytes;
        fence_proxy_async_shared();
        if (cls == 0) {
            band->yoff = 0;
            bytes = (uint32_t)(a.wbox * (a.R + 2) * 16);
            mbar_arrive_expect_tx(mbar, bytes);
            tma_load_3d(stage, map_v, mbar, xc0, ylo, b0);
        } else {
            const int xt = ylo - (((ylo % a.align) + a.align) % a.align);
            band->yoff = ylo - xt;
            bytes = (uint32_t)(a.rbox_h * a.wbox * (int)sizeof(T) * TexelCvt<T>::BG);
            mbar_arrive_expect_tx(mbar, bytes);
            tma_load_3d(stage, map_h, mbar, xt, xc0, b0);
        }
    }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(kFwdThreads, 2) forward_tiled_kernel(const __grid_constant__ CUtensorMap map_v,
                                                                      const __grid_constant__ CUtensorMap map_h,
                                                                      const FwdTiledArgs a) {
    constexpr int BG = TexelCvt<T>::BG;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    int* status = reinterpret_cast<int*>(smem + 16);
    FwdBand* band = reinterpret_cast<FwdBand*>(smem + 32);
    unsigned char* stage = smem + 128;
    uint4* comp = reinterpret_cast<uint4*>(stage + (a.stage_bytes + 127) / 128 * 128);

    const int tid = threadIdx.x;
    const int grp_idx = blockIdx.x / a.n_dr, dr = blockIdx.x - (blockIdx.x / a.n_dr) * a.n_dr;
    const Int2 grp = a.groups[grp_idx];
    const int v0 = grp.x, cnt = grp.y & 0xffff, cls = grp.y >> 16;
    const int d0 = dr * a.Dt;
    const int b0 = blockIdx.y * BG;
    const int vl = tid / a.Dt, d = d0 + (tid - (tid / a.Dt) * a.Dt);
    const bool active = vl < cnt && d < a.D;

    // this thread's ray, in the compute frame (x <-> y swapped for the horizontal class)
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
    int k = 0;
    float acc[BG];
#pragma unroll
    for (int b = 0; b < BG; ++b) acc[b] = 0.0f;

    if (tid == 0) {
        mbar_init(mbar, 1);
        *status = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid < 32) fwd_issue_slab<T>(&map_v, &map_h, a, 0, v0, cnt, cls, d0, b0, mbar, band, stage);

    const int rows = a.R + 2;
    for (int s = 0; s < a.n_slabs; ++s) {
        if (tid == 0) *status = mbar_wait_bounded(mbar, (uint32_t)(s & 1), a.spin_limit) ? 0 : 1;
        __syncthreads();
        if (*status) {
            if (tid == 0) {
                record_device_error(a.err, RADON_ERR_TIMEOUT);
                mbar_wait_bounded(mbar, (uint32_t)(s & 1), a.spin_limit);   // the copy in flight, once more
            }
            return;
        }
        const int xc0 = band->xc0, yoff = band->yoff;
        if (tid == 0 && band->bad) record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
        // ---- repack the staged band into 16-byte texels [row][col][image]
        if (cls == 0) {
            const T* st = reinterpret_cast<const T*>(stage);
            for (int e = tid; e < rows * a.wbox; e += kFwdThreads) {
                const int r = e / a.wbox, c = e - (e / a.wbox) * a.wbox;
                T v[BG];
#pragma unroll
                for (int b = 0; b < BG; ++b) v[b] = st[((size_t)b * rows + r) * a.wbox + c];
                comp[r * a.wc + c] = pack_texel<T>(v);
            }
        } else {
            const T* st = reinterpret_cast<const T*>(stage);
            for (int e = tid; e < rows * a.wbox; e += kFwdThreads) {
                const int c = e / rows, r = e - (e / rows) * rows;
                T v[BG];
#pragma unroll
                for (int b = 0; b < BG; ++b) v[b] = st[((size_t)b * a.wbox + c) * a.rbox_h + yoff + r];
                comp[r * a.wc + c] = pack_texel<T>(v);
            }
        }
        __syncthreads();
        // ---- staging buffer consumed: copy the next slab while this one is projected
        if (tid < 32 && s + 1 < a.n_slabs)
            fwd_issue_slab<T>(&map_v, &map_h, a, s + 1, v0, cnt, cls, d0, b0, mbar, band, stage);
        // ---- march every ray through the slab
        if (k < nk) {
            const int ylo = -3 + s * a.R;
            const float kf = (float)k;
            const float qX = kf * dXh, qY = kf * dYh;   // exact products
            const float QX = floorf(qX), QY = floorf(qY);
            const float sX = fmaf(kf, dXl, fX0 + (qX - QX));
            const float sY = fmaf(kf, dYl, fY0 + (qY - QY));
            const int JB = J0 + (int)QX - xc0;   // band-local integer base of sample k
            const int IB = I0 + (int)QY - ylo;
            // every sample of this slab stays inside the band (the extreme rays' lines enclose the
            // CTA's rays); checked per ray so no access can leave the buffer
            const float ylim = (s == a.n_slabs - 1) ? 3.0e38f : (float)(a.R + 1 - IB);
            // the ray's next sample may lie in a later slab (rays entering through a side)
            const bool here = (sY - 0.5f) < (ylim - 0.5f);
            if (here) {
            const float xa = (float)JB + sX;
            // samples this slab can take: up to the slab end or the ray's last sample, whichever first
            float steps = (float)(nk - 1 - k);
            if (s != a.n_slabs - 1 && fabsf(dY) > 1e-6f * fabsf(dX)) steps = fminf(steps, (ylim - sY) / dY);
            const float xb = fmaf(steps, dX, xa);
            if (fminf(xa, xb) < 1.0f || fmaxf(xa, xb) > (float)(a.wbox - 2) || IB + sY < 0.5f) {
                record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
                k = nk;
            } else {
                // floors by round-to-nearest of (value - 1/2) through the 1.5 * 2^23 magic constant;
                // at exact integers either neighbour gives the same bilinear value
                const float M = 12582912.0f;
                const unsigned magic = 0x4B400000u;
                const float sXm = sX - 0.5f, sYm = sY - 0.5f, ylim_m = ylim - 0.5f;
                const unsigned base = (unsigned)(IB * a.wc + JB) - magic * (unsigned)(a.wc + 1);
                const unsigned wcu = (unsigned)a.wc;
                const int kleft = nk - k;
                int i = 0;
                float kk = 0.0f;
                for (; i < kleft; ++i, kk += 1.0f) {
                    const float fym = fmaf(kk, dY, sYm);
                    if (fym >= ylim_m) break;
                    const float fxm = fmaf(kk, dX, sXm);
                    const float tx = fxm + M, ty = fym + M;
                    const float ax = fxm - (tx - M), ay = fym - (ty - M);   // in [-1/2, 1/2]
                    const unsigned idx = __float_as_uint(ty) * wcu + __float_as_uint(tx) + base;
                    const float wx1 = 0.5f + ax, wx0 = 0.5f - ax, wy1 = 0.5f + ay, wy0 = 0.5f - ay;
                    const float w00 = wx0 * wy0, w01 = wx1 * wy0, w10 = wx0 * wy1, w11 = wx1 * wy1;
                    const uint4* p = comp + idx;
                    float t00[BG], t01[BG], t10[BG], t11[BG];
                    TexelCvt<T>::load(p[0], t00);
                    TexelCvt<T>::load(p[1], t01);
                    TexelCvt<T>::load(p[wcu], t10);
                    TexelCvt<T>::load(p[wcu + 1], t11);
#pragma unroll
                    for (int b = 0; b < BG; ++b)
                        acc[b] = fmaf(w00, t00[b], fmaf(w01, t01[b], fmaf(w10, t10[b], fmaf(w11, t11[b], acc[b]))));
                }
                k += i;
            }
            }
        }
        __syncthreads();
    }
    if (active) {
        T* out = reinterpret_cast<T*>(a.sino);
        const long long vd = (long long)a.V * a.D;
        const long long o = (long long)(v0 + vl) * a.D + d;
#pragma unroll
        for (int b = 0; b < BG; ++b)
            if (b0 + b < a.B) out[(long long)(b0 + b) * vd + o] = from_f32<T>(a.h * acc[b]);
    }
}

}  // namespace radon
