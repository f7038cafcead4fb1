// Tiled gather adjoint (backprojection): x[b][i][j] = h * sum_v sum_d y[b][v][d] * W_vd(i, j), with
// W_vd(i, j) the sum of the bilinear weights that the samples of ray (v, d) put on pixel (i, j).
// The transpose of the forward projection, computed pixel by pixel (no atomics).
//
// One CTA owns a 16 x 16 pixel tile of BG images and loops over every view, so each output
// element is written exactly once.  Views are processed in chunks of kBwdViews:
//   * warp 0 projects the tile onto the detector of each view of chunk c+2 and issues 1-D TMA
//     copies of the needed detector window (every image, every view) into a staging slot;
//   * all threads wait (bounded) for chunk c, convert the window to FP32 image quads
//     ([view][quad][det] float4) and re-base each ray's geometry on the tile origin from the
//     split-precision table (reference sample, step, window constants);
//   * each thread takes its pixel: for every candidate ray (detector index within the projected
//     2x2 support square) it evaluates KW consecutive sample weights in FP32, shared by all BG
//     images, and accumulates weight * y per image.
// Shared-memory image of one CTA (all offsets multiples of 128 B):
//   header      mbarriers, status, per-view window starts / half widths, per-box offsets
//   staging     2 slots x kBwdViews x BG boxes of `stage_stride` bytes (TMA destinations)
//   yq          kBwdViews x NQ x wd float4
//   rp          kBwdViews x wd x 2 float4
#pragma once

#include "device_error.cuh"
#include "dtype.cuh"
#include "epilogue.cuh"
#include "radon_internal.h"
#include "f32x2.cuh"
#include "tma.cuh"

namespace radon {

constexpr int kBwdTile = 16;
constexpr int kBwdThreads = kBwdTile * kBwdTile;
constexpr int kBwdViews = 8;

struct BwdTiledArgs {
    const RayT* rays;
    const int* nks;
    const ViewF* views;
    void* img;
    int n, V, D, B;
    float h;
    int wd;            // detector window per view (>= widest projected tile + slack)
    int wdb;           // TMA box width in elements (wd + alignment)
    int align;         // elements per 16 B
    int stage_stride;  // bytes per staged box (multiple of 128)
    int tiles_x;
    int* err;
    uint32_t spin_limit;
    int stall_test;    // 1: issue no copies (exercises the bounded-wait expiry path)
    int tma_rank;      // 1: 1-D descriptor; 2: the same layout described with a unit outer dimension
    int out_dtype;     // packed variant: storage type of the output image (radon_dtype)
    float ih2;         // packed variant: 1 / h^2 (every ray's step has length h)
    Epilogue ep;
};

__host__ __device__ inline int bwd_nq(int bg) { return (bg + 3) / 4; }

// header: [0,16) mbarriers, [16,20) status, [32,96) window starts [2][8], [96,160) half widths
// [2][8], [160,192) / [192,224) the current chunk's copies, [256, 256 + 64 bg) box offsets [2][8][bg]
__host__ __device__ inline int bwd_header_bytes(int bg) { return ((256 + 64 * bg) + 127) / 128 * 128; }

__host__ __device__ inline size_t bwd_smem_bytes(int bg, int wd, int stage_stride) {
    return 128 + (size_t)bwd_header_bytes(bg) + (size_t)2 * kBwdViews * bg * stage_stride +
           (size_t)kBwdViews * bwd_nq(bg) * wd * 16 + (size_t)kBwdViews * wd * 32;
}

__device__ __forceinline__ float bwd_det_coord(const ViewF& vf, float x, float y) {
    return fmaf(vf.ax, x, fmaf(vf.ay, y, vf.a0)) / fmaf(vf.bx, x, fmaf(vf.by, y, vf.b0));
}

// Detector window of a tile for one view: candidates of every pixel of the tile lie in
// [dlo, floor(tmax + r)], with r the half width of a pixel's 2x2 support square on the detector.
// Parallel beam: r is the constant |ax| + |ay|.  Fan beam: the largest half width at the four tile
// corners, with a 5% margin for its variation across the tile (magnification and ray angle change
// slowly over 16 pixels).  A wider window only adds candidates of weight zero.
__device__ __forceinline__ void bwd_view_window(const ViewF vf, int ti, int tj, int n, int* dlo, float* r_out) {
    const float x0 = (float)tj, x1 = (float)min(tj + kBwdTile - 1, n - 1);
    const float y0 = (float)ti, y1 = (float)min(ti + kBwdTile - 1, n - 1);
    const float t00 = bwd_det_coord(vf, x0, y0), t10 = bwd_det_coord(vf, x1, y0);
    const float t01 = bwd_det_coord(vf, x0, y1), t11 = bwd_det_coord(vf, x1, y1);
    const float tmin = fminf(fminf(t00, t10), fminf(t01, t11));
    float r;
    if (vf.bx == 0.0f && vf.by == 0.0f) {
        r = (fabsf(vf.ax) + fabsf(vf.ay)) / vf.b0;
    } else {
        r = 0.0f;
#pragma unroll
        for (int cidx = 0; cidx < 4; ++cidx) {
            const float cx = (cidx & 1) ? x1 : x0, cy = (cidx & 2) ? y1 : y0;
            const float s0 = bwd_det_coord(vf, cx - 1.0f, cy - 1.0f), s1 = bwd_det_coord(vf, cx + 1.0f, cy - 1.0f);
            const float s2 = bwd_det_coord(vf, cx - 1.0f, cy + 1.0f), s3 = bwd_det_coord(vf, cx + 1.0f, cy + 1.0f);
            r = fmaxf(r, 0.5f * (fmaxf(fmaxf(s0, s1), fmaxf(s2, s3)) - fminf(fminf(s0, s1), fminf(s2, s3))));
        }
        r = fmaf(r, 1.05f, 0.02f);
    }
    r = fmaf(r, 1.0f, 0.01f);
    *dlo = (int)floorf(tmin - r - 0.01f);
    *r_out = r;
}

// Tile-relative parameters of ray (v, d) for the gather: A = (reference sample position relative to
// the tile origin, step), Bq = (step / |step|^2, candidate half-window kr).  The reference sample is
// the one nearest the tile centre (clamped to the ray), re-based from the split-precision table.
// Rays outside the detector or missing the image get a far-away sentinel (weight zero everywhere).
__device__ __forceinline__ void bwd_ray_params(const RayT* rays, const int* nks, int v, int d, int D, int ti, int tj,
                                               float4* A_out, float4* B_out) {
    float4 A = make_float4(1e9f, 1e9f, 0.0f, 0.0f), Bq = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (d >= 0 && d < D) {
        const long long ridx = (long long)v * D + d;
        const int nk = nks[ridx];
        if (nk > 0) {
            const RayT ray = rays[ridx];
            const float dx = ray.dxh + ray.dxl, dy = ray.dyh + ray.dyl;
            const float il = 1.0f / fmaf(dx, dx, dy * dy);
            const float ex = ((float)(tj - ray.J0) + 7.5f) - ray.fx0;
            const float ey = ((float)(ti - ray.I0) + 7.5f) - ray.fy0;
            const float kf = fminf(fmaxf(rintf(fmaf(ex, dx, ey * dy) * il), 0.0f), (float)(nk - 1));
            const float qx = kf * ray.dxh, qy = kf * ray.dyh;   // exact products
            const float Qx = floorf(qx), Qy = floorf(qy);
            A.x = ((float)(ray.J0 - tj) + Qx) + fmaf(kf, ray.dxl, ray.fx0 + (qx - Qx));
            A.y = ((float)(ray.I0 - ti) + Qy) + fmaf(kf, ray.dyl, ray.fy0 + (qy - Qy));
            A.z = dx;
            A.w = dy;
            Bq.x = dx * il;
            Bq.y = dy * il;
            Bq.z = (fabsf(dx) + fabsf(dy)) * il + 1e-4f;
        }
    }
    *A_out = A;
    *B_out = Bq;
}

// Tile-relative position of a ray from its record (already in shared memory): A = (reference sample
// position relative to the tile origin, step).  The sample count is not needed: samples beyond the
// ray's ends lie outside the support box and carry zero weight on every pixel of the image, and a
// ray that misses the image keeps its line (its samples all carry zero weight).  The reference is
// the sample nearest the tile centre, not clamped to the ray: the table keeps k * dxh exact for k up
// to kSplitMarginPx / h samples past either end, which covers every tile the ray's support touches;
// for tiles farther away the products may round, but there every candidate weight is zero.
// Rays outside the detector get a far-away sentinel with step zero (weight zero everywhere).
__device__ __forceinline__ float4 bwd_ray_pos_rec(const RayT ray, bool valid, int ti, int tj, float ih2) {
    float4 A = make_float4(1e9f, 1e9f, 0.0f, 0.0f);
    const float dx = ray.dxh + ray.dxl, dy = ray.dyh + ray.dyl;
    if (valid && (dx != 0.0f || dy != 0.0f)) {
        const float ex = ((float)(tj - ray.J0) + 7.5f) - ray.fx0;
        const float ey = ((float)(ti - ray.I0) + 7.5f) - ray.fy0;
        const float kc = rintf(fmaf(ex, dx, ey * dy) * ih2);
        const float qx = kc * ray.dxh, qy = kc * ray.dyh;
        const float Qx = floorf(qx), Qy = floorf(qy);
        A.x = ((float)(ray.J0 - tj) + Qx) + fmaf(kc, ray.dxl, ray.fx0 + (qx - Qx));
        A.y = ((float)(ray.I0 - ti) + Qy) + fmaf(kc, ray.dyl, ray.fy0 + (qy - Qy));
        A.z = dx;
        A.w = dy;
    }
    return A;
}

// The ray-dependent part of a candidate window's start, hoisted out of the per-pixel work:
// kap - kr = (p - A).b - kr = p.b + C with b = step / |step|^2 and C = -A.b - kr (a sentinel ray
// has step zero, so C = -1e-4 and every weight stays zero).
__device__ __forceinline__ float bwd_ray_window_c(const float4 A, float ih2) {
    const float bx = A.z * ih2, by = A.w * ih2;
    const float kr = fmaf(fabsf(A.z) + fabsf(A.w), ih2, 1e-4f);
    return -fmaf(A.x, bx, A.y * by) - kr;
}

// Bilinear weight of the pixel at p2 (tile-local) on the ray with tile-relative reference sample a0
// and step d2: the sum over the KW samples from the window start ceil(p.b + C) (C from
// bwd_ray_window_c), each a product of two tents.  The x and y halves run as f32x2 pairs.
template <int KW>
__device__ __forceinline__ float bwd_ray_weight_c(f32x2 p2, float px, float py, f32x2 a0, f32x2 d2, f32x2 ih2_2,
                                                  float C) {
    const f32x2 e2 = f2_sub(a0, p2);   // A - p
    float bx, by;
    f2_unpack(f2_mul(d2, ih2_2), &bx, &by);
    const float ka = ceilf(fmaf(px, bx, fmaf(py, by, C)));
    f32x2 r2 = f2_fma(f2_pack(ka, ka), d2, e2);   // ka * step - (p - A)
    float w = 0.0f;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        float rx, ry;
        f2_unpack(r2, &rx, &ry);
        const float wx = fmaxf(0.0f, 1.0f - fabsf(rx));
        const float wy = fmaxf(0.0f, 1.0f - fabsf(ry));
        w = fmaf(wx, wy, w);
        if (k + 1 < KW) r2 = f2_add(r2, d2);
    }
    return w;
}

// Warp 0: windows for the views of chunk c and the TMA copies into staging slot `slot`.
template <typename T, int BG>
__device__ void bwd_issue_chunk(const CUtensorMap* tmap, const BwdTiledArgs& a, int c, int slot, int ti, int tj,
                                int b0, uint64_t* mbar, int* dlo_s, float* r_s, int* off_s, unsigned char* stage) {
    const int lane = threadIdx.x & 31;
    const int v0 = c * kBwdViews;
    const int nv = min(kBwdViews, a.V - v0);
    if (lane < nv) {
        int dlo;
        float r;
        bwd_view_window(a.views[v0 + lane], ti, tj, a.n, &dlo, &r);
        dlo_s[slot * kBwdViews + lane] = dlo;
        r_s[slot * kBwdViews + lane] = r;
    }
    __syncwarp();
    if (a.stall_test) return;   // no copies: the wait on this slot must expire
    if (lane == 0) {
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&mbar[slot], (uint32_t)(nv * BG * a.wdb * (int)sizeof(T)));
    }
    __syncwarp();
    for (int e = lane; e < nv * BG; e += 32) {
        const int vl = e / BG, b = e - (e / BG) * BG;
        const long long x = (long long)(b0 + b) * a.V * a.D + (long long)(v0 + vl) * a.D + dlo_s[slot * kBwdViews + vl];
        const long long xs = x - (((x % a.align) + a.align) % a.align);   // floor to a 16 B boundary
        off_s[(slot * kBwdViews + vl) * BG + b] = (int)(x - xs);
        unsigned char* dst = stage + ((size_t)(slot * kBwdViews + vl) * BG + b) * a.stage_stride;
        if (a.tma_rank == 1)
            tma_load_1d(dst, tmap, &mbar[slot], (int)xs);
        else
            tma_load_2d(dst, tmap, &mbar[slot], (int)xs, 0);
    }
}

template <int KW>
__device__ __forceinline__ float bwd_ray_weight(float px, float py, const float4 A, const float4 Bq) {
    // A = (rx, ry, dx, dy): reference sample position (tile-local) and step; Bq = (dx il, dy il, kr, -)
    const float ex = px - A.x, ey = py - A.y;
    const float kap = fmaf(ex, Bq.x, ey * Bq.y);
    const float ka = ceilf(kap - Bq.z);
    float rx = fmaf(ka, A.z, -ex), ry = fmaf(ka, A.w, -ey);
    float w = 0.0f;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        const float wx = fmaxf(0.0f, 1.0f - fabsf(rx));
        const float wy = fmaxf(0.0f, 1.0f - fabsf(ry));
        w = fmaf(wx, wy, w);
        rx += A.z;
        ry += A.w;
    }
    return w;
}

template <typename T, int BG, int KW>
__global__ void __launch_bounds__(kBwdThreads, 2) backward_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                       const BwdTiledArgs a) {
    constexpr int NQ = (BG + 3) / 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations need 128 B alignment: round the dynamic base up (the size includes 128 B slack)
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    int* status = reinterpret_cast<int*>(smem + 16);
    int* dlo_s = reinterpret_cast<int*>(smem + 32);               // [2][V]
    float* r_s = reinterpret_cast<float*>(smem + 32 + 64);        // [2][V]
    int* dlo_c = reinterpret_cast<int*>(smem + 32 + 128);         // [V]
    float* r_c = reinterpret_cast<float*>(smem + 32 + 160);       // [V]
    int* off_s = reinterpret_cast<int*>(smem + 256);              // [2][V][BG]
    unsigned char* stage = smem + bwd_header_bytes(BG);
    const size_t slot_bytes = (size_t)kBwdViews * BG * a.stage_stride;
    float4* yq = reinterpret_cast<float4*>(stage + 2 * slot_bytes);
    float4* rp = yq + kBwdViews * NQ * a.wd;

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int ti = (tile / a.tiles_x) * kBwdTile, tj = (tile - (tile / a.tiles_x) * a.tiles_x) * kBwdTile;
    const int b0 = blockIdx.y * BG;
    const int nchunks = (a.V + kBwdViews - 1) / kBwdViews;
    const int pi = tid / kBwdTile, pj = tid - (tid / kBwdTile) * kBwdTile;
    const float px = (float)pj, py = (float)pi;            // tile-local pixel coordinates
    const float gx = (float)(tj + pj), gy = (float)(ti + pi);
    const bool inside = (ti + pi) < a.n && (tj + pj) < a.n;

    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        *status = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid < 32) {
        bwd_issue_chunk<T, BG>(&tmap, a, 0, 0, ti, tj, b0, mbar, dlo_s, r_s, off_s, stage);
        if (nchunks > 1) bwd_issue_chunk<T, BG>(&tmap, a, 1, 1, ti, tj, b0, mbar, dlo_s, r_s, off_s, stage);
    }

    float acc[BG];
#pragma unroll
    for (int b = 0; b < BG; ++b) acc[b] = 0.0f;

    for (int c = 0; c < nchunks; ++c) {
        const int slot = c & 1;
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        const int v0 = c * kBwdViews;
        const int nv = min(kBwdViews, a.V - v0);
        if (tid == 0) *status = mbar_wait_bounded(&mbar[slot], parity, a.spin_limit) ? 0 : 1;
        __syncthreads();
        if (*status) {
            if (tid == 0) {
                record_device_error(a.err, RADON_ERR_TIMEOUT);
                // let any copy still in flight into the other slot land before the CTA exits
                if (c + 1 < nchunks && !a.stall_test)
                    mbar_wait_bounded(&mbar[slot ^ 1], (uint32_t)(((c + 1) >> 1) & 1), a.spin_limit);
            }
            return;
        }
        // ---- repack the staged windows and re-base the rays on the tile origin
        for (int e = tid; e < nv * a.wd; e += kBwdThreads) {
            const int vl = e / a.wd, dl = e - (e / a.wd) * a.wd;
            const int v = v0 + vl;
            const int dlo = dlo_s[slot * kBwdViews + vl];
            const int d = dlo + dl;
            const T* box0 = reinterpret_cast<const T*>(stage + (size_t)(slot * kBwdViews + vl) * BG * a.stage_stride);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float vals[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int b = 4 * q + u;
                    if (b < BG) {
                        const T* box = reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(box0) +
                                                                  (size_t)b * a.stage_stride);
                        vals[u] = to_f32(box[off_s[(slot * kBwdViews + vl) * BG + b] + dl]);
                    } else {
                        vals[u] = 0.0f;
                    }
                }
                yq[(vl * NQ + q) * a.wd + dl] = make_float4(vals[0], vals[1], vals[2], vals[3]);
            }
            float4 A, Bq;
            bwd_ray_params(a.rays, a.nks, v, d, a.D, ti, tj, &A, &Bq);
            rp[(vl * a.wd + dl) * 2] = A;
            rp[(vl * a.wd + dl) * 2 + 1] = Bq;
        }
        if (tid < nv) {
            dlo_c[tid] = dlo_s[slot * kBwdViews + tid];
            r_c[tid] = r_s[slot * kBwdViews + tid];
        }
        __syncthreads();
        // ---- staging slot consumed: start the copies of chunk c + 2 into it
        if (tid < 32 && c + 2 < nchunks)
            bwd_issue_chunk<T, BG>(&tmap, a, c + 2, slot, ti, tj, b0, mbar, dlo_s, r_s, off_s, stage);
        // ---- gather
        for (int vl = 0; vl < nv; ++vl) {
            const ViewF vf = a.views[v0 + vl];
            const int dlo = dlo_c[vl];
            const float r = r_c[vl];
            const float t = bwd_det_coord(vf, gx, gy);
            const float flo = ceilf(t - r), fhi = floorf(t + r);
            int da = (int)fmaxf(flo, (float)max(dlo, 0));
            int db = (int)fminf(fhi, (float)min(a.D - 1, dlo + a.wd - 1));
            if (inside && ((flo < (float)dlo && flo >= 0.0f) || (fhi > (float)(dlo + a.wd - 1) && fhi <= (float)(a.D - 1))))
                record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
            const float4* rpv = rp + vl * a.wd * 2;
            const float4* yqv = yq + vl * NQ * a.wd;
            for (int d = da; d <= db; ++d) {
                const int dl = d - dlo;
                const float w = bwd_ray_weight<KW>(px, py, rpv[dl * 2], rpv[dl * 2 + 1]);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 y4 = yqv[q * a.wd + dl];
                    if (4 * q + 0 < BG) acc[4 * q + 0] = fmaf(w, y4.x, acc[4 * q + 0]);
                    if (4 * q + 1 < BG) acc[4 * q + 1] = fmaf(w, y4.y, acc[4 * q + 1]);
                    if (4 * q + 2 < BG) acc[4 * q + 2] = fmaf(w, y4.z, acc[4 * q + 2]);
                    if (4 * q + 3 < BG) acc[4 * q + 3] = fmaf(w, y4.w, acc[4 * q + 3]);
                }
            }
        }
        __syncthreads();
    }
    if (inside) {
        T* out = reinterpret_cast<T*>(a.img);
        const long long npix = (long long)a.n * a.n;
        const long long p = (long long)(ti + pi) * a.n + (tj + pj);
#pragma unroll
        for (int b = 0; b < BG; ++b)
            if (b0 + b < a.B) {
                const long long idx = (long long)(b0 + b) * npix + p;
                out[idx] = from_f32<T>(epilogue_value<T>(a.ep, a.h * acc[b], idx));
            }
    }
}


}  // namespace radon
