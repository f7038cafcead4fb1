// Uneven batches in one persistent launch: many images of different sizes, each with its own
// geometry (Section 4.1's batch processing, generalised to a mixed batch).
//
// A plan turns every image of every item into a unit and every unit into work items -- blocks of
// rays for the forward projection, 16 x 16 pixel tiles for the adjoint -- listed largest first.  One
// persistent kernel (as many CTAs as fit on the GPU at once) takes work items from a device counter
// until the list is exhausted, so a 1024^2 image with 1000 views and a 128^2 image with 90 views
// share the SMs without a tail.  Items have batch 1 in the typical mixed batch, so nothing is
// amortised across images as in the batch-interleaved kernels; instead:
//   * forward: a pack kernel stores each pixel's 2 x 2 bilinear neighbourhood as one texel (four
//     16-bit values in 8 bytes, or four FP32 in 16), once in the image frame and once transposed;
//     every sample is one texel load through L1.  Four lanes share a ray (interleaved samples,
//     partial sums joined by a fixed shuffle tree) and a warp holds eight neighbouring detectors of
//     one view, whose samples at a given step lie along the detector direction; the frame whose rows
//     run along that direction keeps them within a few cache lines;
//   * adjoint: per chunk of views the CTA computes each view's detector window for its tile and
//     stages the window's sinogram values in shared memory; then every thread gathers its pixel
//     from shared memory.  For a parallel-beam view every ray shares one sample lattice, so the CTA
//     re-bases one ray per view and each pixel steps from one candidate ray's samples to the
//     next; a fan-beam view re-bases every ray of its window (one ray per thread).
// Tile shapes (forward: views x detectors per ray block; adjoint: views per chunk) are chosen per
// image size by timing each candidate on the plan's own buffers when the plan is created.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "backward_tiled.cuh"
#include "device_error.cuh"
#include "dtype.cuh"
#include "epilogue.cuh"
#include "radon_internal.h"
#include "tma.cuh"

namespace radon {

namespace {

constexpr uint64_t kPlanMagic = 0x5241444f4e504c4eULL;   // "RADONPLN"
constexpr int kPlanThreads = 256;
constexpr int kMaxChunkViews = 32;   // adjoint: views per staged chunk at most (16 where 32 do not fit)

struct Unit {
    const void* in;
    void* out;
    const RayT* rays;
    const int* nks;
    const ViewF* views;
    long long q_off;   // forward: first texel of this unit's packed image (row frame; transposed follows)
    int n, V, D;
    float h, ih2;
    int wd;            // adjoint: detector window of a 16 x 16 tile
    int cfg;           // forward: views per ray block; adjoint: views per chunk
    int lanes;         // forward: lanes per ray (1 or 4)
    int fan;           // 1: fan beam (detector coordinate a ratio); 0: parallel (affine)
    int cand3;         // adjoint, parallel beam: every pixel's candidate window holds at most 3 rays
    const Int2* groups;   // forward, staged: view groups of one orientation class for G = cfg
    int n_groups;
    int R;                // forward, staged: texel rows per slab
    int staged;           // forward: 1 = the staged kernel, 0 = the L1 gather
};

struct Work {
    int unit;
    int tile;
};

// ------------------------------------------------------------------------------------------ pack

template <typename T>
struct Quad;   // texel: the 2 x 2 neighbourhood (i, j), (i, j+1), (i+1, j), (i+1, j+1)

template <>
struct Quad<float> {
    using type = float4;
    __device__ static type make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
    __device__ static void unpack(const type& q, float* v) {
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    }
};

template <typename H>
struct Quad16 {
    using type = uint2;
    __device__ static unsigned bits(H v) {
        unsigned short u;
        memcpy(&u, &v, 2);
        return u;
    }
    __device__ static type make(H a, H b, H c, H d) {
        return make_uint2(bits(a) | (bits(b) << 16), bits(c) | (bits(d) << 16));
    }
};

template <>
struct Quad<__half> : Quad16<__half> {
    __device__ static void unpack(const type& q, float* v) {
        __half2 lo, hi;
        memcpy(&lo, &q.x, 4);
        memcpy(&hi, &q.y, 4);
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
};

template <>
struct Quad<__nv_bfloat16> : Quad16<__nv_bfloat16> {
    __device__ static void unpack(const type& q, float* v) {
        v[0] = __uint_as_float(q.x << 16);
        v[1] = __uint_as_float(q.x & 0xffff0000u);
        v[2] = __uint_as_float(q.y << 16);
        v[3] = __uint_as_float(q.y & 0xffff0000u);
    }
};

template <typename T>
__device__ __forceinline__ T pix(const T* x, int n, int i, int j) {
    return (i >= 0 && i < n && j >= 0 && j < n) ? x[(long long)i * n + j] : from_f32<T>(0.0f);
}

}  // namespace
}  // namespace radon

#include "staged_forward.cuh"

namespace radon {
namespace {

// ------------------------------------------------------------------------------------- forward

// Lanes per ray of the forward work items (a tuned shape: 1 or 4).  With four, the lanes of a ray take
// its samples k = sub, sub + 4, ... (spatially neighbouring texels, so a warp's loads stay within a
// few cache lines), which gives the SM four times the independent loads in flight -- the shape for
// images whose rays alone do not fill the GPU -- and sum their partial sums in a fixed shuffle tree
// (the same bits on every call).
constexpr int kPlanMaxLanes = 4;

// Ray (v, d) of unit u, lane `sub` of its group: the partial sum over its samples (without the factor
// h), every sample one texel load.  Positions are re-based from the split-precision table every 32 samples.
template <typename T>
__device__ float plan_ray(const Unit& u, const typename Quad<T>::type* __restrict__ quads, int v, int d, int sub,
                          int lanes) {
    const long long r = (long long)v * u.D + d;
    const int nk = u.nks[r];
    if (nk == 0) return 0.0f;
    const RayT ray = u.rays[r];
    // frame: rows of the transposed image for rays running mostly along x (neighbouring rays then
    // differ mostly in y, which the transposed frame lays out along its rows)
    const bool tr = fabsf(ray.dxh + ray.dxl) > fabsf(ray.dyh + ray.dyl);
    const int J0 = tr ? ray.I0 : ray.J0, I0 = tr ? ray.J0 : ray.I0;
    const float fX0 = tr ? ray.fy0 : ray.fx0, fY0 = tr ? ray.fx0 : ray.fy0;
    const float dXh = tr ? ray.dyh : ray.dxh, dYh = tr ? ray.dxh : ray.dyh;
    const float dXl = tr ? ray.dyl : ray.dxl, dYl = tr ? ray.dxl : ray.dyl;
    const float dX = dXh + dXl, dY = dYh + dYl;
    const int p = sq_pitch(u.n);
    const typename Quad<T>::type* q = quads + u.q_off + (tr ? sq_frame(u.n) : 0ll);
    const unsigned last = (unsigned)sq_frame(u.n) - 1u;
    const float M = 12582912.0f;          // 1.5 * 2^23: x + M rounds x to the nearest integer
    const unsigned magic = 0x4B400000u;   // the bit pattern of M
    float acc = 0.0f;
    for (int kb = 0; kb < nk; kb += 32) {
        const float kbf = (float)kb;
        const float qx = kbf * dXh, qy = kbf * dYh;   // exact products
        const float QX = floorf(qx), QY = floorf(qy);
        const float sXm = fmaf(kbf, dXl, fX0 + (qx - QX)) - 0.5f;
        const float sYm = fmaf(kbf, dYl, fY0 + (qy - QY)) - 0.5f;
        const int jb = J0 + (int)QX, ib = I0 + (int)QY;
        // texel index of a sample: (ib + floor(ly) + 2) p + (jb + floor(lx) + 2), each floor taken as
        // the nearest integer to (l - 1/2) through the magic constant, whose bias cancels modulo 2^32
        // (at an exact integer either neighbour gives the same bilinear value)
        const unsigned base = (unsigned)((ib + 2) * p + (jb + 2)) - magic * (unsigned)(p + 1);
        const int kend = min(nk - kb, 32);
#pragma unroll 1   // unrolled loops measured slower (registers)
        for (int kk = sub; kk < kend; kk += lanes) {
            const float fxm = fmaf((float)kk, dX, sXm), fym = fmaf((float)kk, dY, sYm);
            const float tx = fxm + M, ty = fym + M;
            // samples lie strictly inside the support box, so every texel index is in range; FP32
            // rounding within ~1e-5 px of the box edge may step one texel past the border, where the
            // weight is ~0: the clamp keeps every read inside the texel array
            const unsigned idx = min(__float_as_uint(ty) * (unsigned)p + __float_as_uint(tx) + base, last);
            const float a = (fxm - (tx - M)) + 0.5f, b = (fym - (ty - M)) + 0.5f;   // fractions in [0, 1]
            float t[4];
            Quad<T>::unpack(__ldg(q + idx), t);   // one 8/16-byte load
            const float top = fmaf(a, t[1] - t[0], t[0]), bot = fmaf(a, t[3] - t[2], t[2]);
            acc += fmaf(b, bot - top, top);
        }
    }
    return acc;
}

// Work item `tile` of unit u (a block of G views x 256 / (G lanes) detectors, `lanes` lanes per ray),
// stored through the epilogue (the identity for plans).  Every thread of the CTA calls it (the lanes
// of a ray meet in shuffles).
template <typename T>
__device__ __forceinline__ void plan_forward_tile(const Unit& u, int tile, const typename Quad<T>::type* __restrict__ quads,
                                                  const Epilogue& ep) {
    const int lanes = u.lanes;
    const int G = u.cfg, Dt = kPlanThreads / (lanes * G);
    const int n_dr = (u.D + Dt - 1) / Dt;
    const int vg = tile / n_dr, dr = tile - (tile / n_dr) * n_dr;
    const int tid = (int)threadIdx.x;
    int vl, dl, sub = 0;
    if (lanes == kPlanMaxLanes) {
        const int ray = tid >> 2;
        sub = tid & 3;
        vl = ray / Dt;
        dl = ray - vl * Dt;
    } else if (G >= 2) {
        // one lane per ray: each group of eight lanes takes views 2m, 2m + 1 x four consecutive
        // detectors, whose quads' cache lines overlap more than those of eight detectors of one view
        // (1-4 % faster from 60 to 1024 views; lane pairs still hold neighbouring detectors)
        const int per = Dt >> 2, P = tid >> 3;
        vl = (P / per) * 2 + ((tid >> 2) & 1);
        dl = (P - (P / per) * per) * 4 + (tid & 3);
    } else {
        vl = tid / Dt;
        dl = tid - vl * Dt;
    }
    const int v = vg * G + vl, d = dr * Dt + dl;
    const bool live = v < u.V && d < u.D;
    float y = live ? plan_ray<T>(u, quads, v, d, sub, lanes) : 0.0f;
    if (lanes == kPlanMaxLanes) {   // uniform over the CTA: one work item at a time
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        y += __shfl_xor_sync(0xffffffffu, y, 2);
    }
    if (live && sub == 0) {
        const long long idx = (long long)v * u.D + d;
        static_cast<T*>(u.out)[idx] = from_f32<T>(epilogue_value<T>(ep, u.h * y, idx));
    }
}

template <typename T>
__global__ void __launch_bounds__(kPlanThreads) plan_forward_kernel(const Unit* __restrict__ units,
                                                                    const Work* __restrict__ work, int n_work,
                                                                    unsigned* counter,
                                                                    const typename Quad<T>::type* __restrict__ quads) {
    __shared__ int s_w;
    for (;;) {
        if (threadIdx.x == 0) s_w = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int wi = s_w;
        __syncthreads();
        if (wi >= n_work) return;
        const Work w = work[wi];
        plan_forward_tile<T>(units[w.unit], w.tile, quads, Epilogue{1.0f, nullptr, 0.0f, nullptr});
    }
}

// Single image (a batch-1 call): the same work items, one CTA each, the unit passed by value.
template <typename T>
__global__ void __launch_bounds__(kPlanThreads) single_forward_kernel(const Unit u,
                                                                      const typename Quad<T>::type* __restrict__ quads,
                                                                      const Epilogue ep) {
    plan_forward_tile<T>(u, (int)blockIdx.x, quads, ep);
}

// ------------------------------------------------------------------------------------- adjoint

struct AdjShared {
    ViewF view[kMaxChunkViews];
    int dlo[kMaxChunkViews];
    float r[kMaxChunkViews];
    // parallel beams: the window's first ray's sample nearest the tile centre (tile-relative) and
    // step, the offset between neighbouring rays' samples of one lattice index, and the window
    // constants (step / h^2, C) of the candidate samples
    float4 ref[kMaxChunkViews];
    float4 bc[kMaxChunkViews];   // (bx, by, C, -)
    float2 dn[kMaxChunkViews];
    int w;
};

// Staging buffers of the adjoint's view chunks in dynamic shared memory.
struct AdjBuffers {
    AdjShared* sh;
    float4* rp;   // [chunk * wd] re-based ray positions and steps
    float* ys;    // [chunk * wd] sinogram values
    float* rc;    // [chunk * wd] window constants
};

// `cap` views per chunk at most, `max_wd` rays per view window.
__device__ __forceinline__ AdjBuffers adj_buffers(unsigned char* smem_raw, int max_wd, int cap) {
    AdjBuffers b;
    b.sh = reinterpret_cast<AdjShared*>(smem_raw);
    b.rp = reinterpret_cast<float4*>(smem_raw + (sizeof(AdjShared) + 15) / 16 * 16);
    b.ys = reinterpret_cast<float*>(b.rp + cap * max_wd);
    b.rc = b.ys + cap * max_wd;
    return b;
}

// Work item `tile` of unit u (a 16 x 16 pixel tile over all views), stored through the epilogue
// (the identity for plans).  Every thread of the CTA calls it (it holds CTA barriers).  FAN = u.fan:
// a parallel-beam view's detector coordinate is affine in the pixel (denominator 1), so its division
// is left out (the same bits: the approximate quotient by 1 is exact).
template <typename T, int KW, bool FAN>
__device__ void plan_adjoint_tile(const Unit& u, int tile, const AdjBuffers& b, const Epilogue& ep, int* err) {
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // 4 x 8 pixels per warp, each group of eight lanes (one 16-byte shared-load phase) a 4 x 2 block
    const int pi = (warp >> 1) * 4 + ((lane & 7) >> 1), pj = (warp & 1) * 8 + (lane >> 3) * 2 + (lane & 1);
    const f32x2 p2 = f2_pack((float)pj, (float)pi);
    const int tiles_x = (u.n + kBwdTile - 1) / kBwdTile;
    const int ti = (tile / tiles_x) * kBwdTile, tj = (tile - (tile / tiles_x) * tiles_x) * kBwdTile;
    const float gx = (float)(tj + pj), gy = (float)(ti + pi);
    const bool inside = (ti + pi) < u.n && (tj + pj) < u.n;
    const f32x2 ih2_2 = f2_pack(u.ih2, u.ih2);
    const T* y = static_cast<const T*>(u.in);
    const int CV = u.cfg, wd = u.wd;
    float acc = 0.0f;
    bool viol = false;
    for (int c0 = 0; c0 < u.V; c0 += CV) {
        const int nv = min(CV, u.V - c0);
        if (tid < nv) {
            const ViewF vf = u.views[c0 + tid];
            int dlo;
            float r;
            bwd_view_window(vf, ti, tj, u.n, &dlo, &r);
            b.sh->view[tid] = vf;
            b.sh->dlo[tid] = dlo;
            b.sh->r[tid] = r;
        }
        __syncthreads();
        for (int e = tid; e < nv * wd; e += kPlanThreads) {
            const int vl = e / wd, dl = e - (e / wd) * wd;
            const int d = b.sh->dlo[vl] + dl;
            const bool valid = d >= 0 && d < u.D;
            const long long ridx = (long long)(c0 + vl) * u.D + (valid ? d : 0);
            const RayT ray = u.rays[ridx];
            const float4 A = bwd_ray_pos_rec(ray, valid, ti, tj, u.ih2);
            b.rp[e] = A;
            b.rc[e] = bwd_ray_window_c(A, u.ih2);
            b.ys[e] = valid ? to_f32(y[ridx]) : 0.0f;
        }
        __syncthreads();
        for (int vl = 0; vl < nv; ++vl) {
            const ViewF vf = b.sh->view[vl];
            const int dlo = b.sh->dlo[vl];
            const float r = b.sh->r[vl];
            const float num = fmaf(vf.ax, gx, fmaf(vf.ay, gy, vf.a0));
            const float t = FAN ? __fdividef(num, fmaf(vf.bx, gx, fmaf(vf.by, gy, vf.b0))) : num;
            const float flo = ceilf(t - r), fhi = floorf(t + r);
            const int da = (int)fmaxf(flo, (float)max(dlo, 0));
            const int db = (int)fminf(fhi, (float)min(u.D - 1, dlo + wd - 1));
            // a window that misses a candidate is reported once per pixel, after the views
            viol |= (flo < (float)dlo && flo >= 0.0f) || (fhi > (float)(dlo + wd - 1) && fhi <= (float)(u.D - 1));
            const ulonglong2* rpv = reinterpret_cast<const ulonglong2*>(b.rp) + vl * wd;
            const float* yv = b.ys + vl * wd;
            const float* cv = b.rc + vl * wd;
            for (int d = da; d <= db; ++d) {
                const ulonglong2 rr = rpv[d - dlo];
                acc = fmaf(bwd_ray_weight_c<KW>(p2, (float)pj, (float)pi, rr.x, rr.y, ih2_2, cv[d - dlo]), yv[d - dlo], acc);
            }
        }
        __syncthreads();
    }
    if (inside && viol) record_device_error(err, RADON_ERR_DEVICE_BOUNDS);
    if (inside) {
        const long long idx = (long long)(ti + pi) * u.n + (tj + pj);
        static_cast<T*>(u.out)[idx] = from_f32<T>(epilogue_value<T>(ep, u.h * acc, idx));
    }
}

// Parallel beams: every ray of a view has the same direction and the rays' sample lattices line up
// (sample k of ray d sits at m_d + k h u with m_d = s_d n, so sample k of ray d + 1 is sample k of
// ray d moved by det_spacing * n).  So the CTA re-bases one ray per view -- the window's first --
// and stages only the window's sinogram values; each pixel finds its first candidate sample ka once
// per view (the same lattice index on every ray) and steps from one candidate ray to the next by
// det_spacing * n.  Every lattice point within a pixel's 2 x 2 support lies inside the support box,
// so it is a sample of its ray whenever the ray exists; rays outside the detector have zero values.
// NC > 0: every candidate window [t - r, t + r] is shorter than NC rays and the staged window holds
// at least NC, so each pixel steps through exactly NC rays from its first candidate (moved back
// inside the window at its end), unrolled; rays beyond the pixel's support square carry weight zero
// and add nothing.  NC = 0: a loop over the pixel's candidates.
template <typename T, int KW, int NC>
__device__ void plan_adjoint_tile_parallel(const Unit& u, int tile, const AdjBuffers& b, const Epilogue& ep,
                                           int* err) {
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // 4 x 8 pixels per warp, each group of eight lanes (one shared-load phase) a 4 x 2 block
    const int pi = (warp >> 1) * 4 + ((lane & 7) >> 1), pj = (warp & 1) * 8 + (lane >> 3) * 2 + (lane & 1);
    const float px = (float)pj, py = (float)pi;
    const int tiles_x = (u.n + kBwdTile - 1) / kBwdTile;
    const int ti = (tile / tiles_x) * kBwdTile, tj = (tile - (tile / tiles_x) * tiles_x) * kBwdTile;
    const float gx = (float)(tj + pj), gy = (float)(ti + pi);
    const T* y = static_cast<const T*>(u.in);
    const int CV = u.cfg, wd = u.wd;
    const float inv_wd = 1.0f / (float)wd, wd_last = (float)(wd - 1);
    const uint32_t ys_a = smem_u32(b.ys);
    float acc = 0.0f;
    for (int c0 = 0; c0 < u.V; c0 += CV) {
        const int nv = min(CV, u.V - c0);
        if (tid < nv) {
            ViewF vf = u.views[c0 + tid];
            int dlo;
            float r;
            bwd_view_window(vf, ti, tj, u.n, &dlo, &r);
            // every pixel's candidates [ceil(t - r), floor(t + r)] within the detector must lie in the
            // staged window (the tile's largest t is at a corner); the loop clamps to it, so a miss is
            // recorded, not overrun
            const float x1 = (float)min(tj + kBwdTile - 1, u.n - 1), y1 = (float)min(ti + kBwdTile - 1, u.n - 1);
            const float tmax = fmaxf(fmaxf(bwd_det_coord(vf, (float)tj, (float)ti), bwd_det_coord(vf, x1, (float)ti)),
                                     fmaxf(bwd_det_coord(vf, (float)tj, y1), bwd_det_coord(vf, x1, y1)));
            if (fminf(floorf(tmax + r), (float)(u.D - 1)) > (float)(dlo + wd - 1)) record_device_error(err, RADON_ERR_DEVICE_BOUNDS);
            // every ray keeps its line in the table (a ray missing the image included)
            const int dref = min(max(dlo, 0), u.D - 1);
            const float4 A = bwd_ray_pos_rec(u.rays[(long long)(c0 + tid) * u.D + dref], true, ti, tj, u.ih2);
            // det_spacing * n = (ax, ay) / (ax^2 + ay^2): the map t = (n.P) / det_spacing + const
            const float q = 1.0f / fmaf(vf.ax, vf.ax, vf.ay * vf.ay);
            const float2 dn = make_float2(vf.ax * q, vf.ay * q);
            const float bx = A.z * u.ih2, by = A.w * u.ih2;
            const float kr = fmaf(fabsf(A.z) + fabsf(A.w), u.ih2, 1e-4f);
            const float sh = (float)(dlo - dref);
            vf.a0 -= (float)dlo;   // window-relative detector coordinate
            b.sh->view[tid] = vf;
            b.sh->dlo[tid] = dlo;
            b.sh->r[tid] = r;
            b.sh->ref[tid] = make_float4(fmaf(sh, dn.x, A.x), fmaf(sh, dn.y, A.y), A.z, A.w);
            b.sh->bc[tid] = make_float4(bx, by, -fmaf(A.x, bx, A.y * by) - kr, 0.0f);
            b.sh->dn[tid] = dn;
        }
        __syncthreads();
        for (int e = tid; e < nv * wd; e += kPlanThreads) {
            int vl = (int)((float)e * inv_wd);   // e / wd, corrected for the quotient's rounding
            vl -= vl * wd > e;
            vl += (vl + 1) * wd <= e;
            const int d = b.sh->dlo[vl] + (e - vl * wd);
            b.ys[e] = (d >= 0 && d < u.D) ? to_f32(y[(long long)(c0 + vl) * u.D + d]) : 0.0f;
        }
        __syncthreads();
        for (int vl = 0; vl < nv; ++vl) {
            const float4 vf0 = *reinterpret_cast<const float4*>(&b.sh->view[vl]);   // ax, ay, a0 - dlo, -
            const float r = b.sh->r[vl];
            const float t = fmaf(vf0.x, gx, fmaf(vf0.y, gy, vf0.z));
            // window-relative candidate range, clamped in FP32 (a non-finite coordinate still gives a
            // loop inside the window)
            const int la0 = __float2int_ru(fmaxf(t - r, 0.0f));
            const int la = NC > 0 ? min(la0, wd - NC) : la0;
            const float4 A = b.sh->ref[vl];
            const float4 bc = b.sh->bc[vl];
            const float2 dn = b.sh->dn[vl];
            const float ka = ceilf(fmaf(px, bc.x, fmaf(py, bc.y, bc.z)));
            const float fla = (float)la;
            // sample ka of the first candidate ray, relative to the pixel
            // (x, y) pairs advance as f32x2 (one instruction per pair); the tents stay scalar
            f32x2 r2 = f2_pack(fmaf(ka, A.z, fmaf(fla, dn.x, A.x) - px), fmaf(ka, A.w, fmaf(fla, dn.y, A.y) - py));
            const f32x2 st2 = f2_pack(A.z, A.w), dn2 = f2_pack(dn.x, dn.y);
            uint32_t ya = ys_a + (uint32_t)(vl * wd + la) * 4u;
            // one candidate ray: its KW samples' weights against the pixel, times the ray's value
            auto candidate = [&]() {
                f32x2 s2 = r2;
                float sx, sy;
                f2_unpack(s2, &sx, &sy);
                float w = __saturatef(1.0f - fabsf(sx)) * __saturatef(1.0f - fabsf(sy));
#pragma unroll
                for (int k = 1; k < KW; ++k) {
                    s2 = f2_add(s2, st2);
                    f2_unpack(s2, &sx, &sy);
                    w = fmaf(__saturatef(1.0f - fabsf(sx)), __saturatef(1.0f - fabsf(sy)), w);
                }
                float yv;
                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(yv) : "r"(ya));
                acc = fmaf(w, yv, acc);
                r2 = f2_add(r2, dn2);
                ya += 4u;
            };
            if constexpr (NC > 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) candidate();
            } else {
                const int lb = __float2int_rd(fminf(t + r, wd_last));
                for (int l = la; l <= lb; ++l) candidate();
            }
        }
        __syncthreads();
    }
    if ((ti + pi) < u.n && (tj + pj) < u.n) {
        const long long idx = (long long)(ti + pi) * u.n + (tj + pj);
        static_cast<T*>(u.out)[idx] = from_f32<T>(epilogue_value<T>(ep, u.h * acc, idx));
    }
}

// Four CTAs per SM: with both geometry kinds in one kernel the register allocation would otherwise
// drop it to three (8.6 % slower on the uneven batch; 1.4 % faster than one generic path at four).
template <typename T, int KW>
__global__ void __launch_bounds__(kPlanThreads, 4) plan_adjoint_kernel(const Unit* __restrict__ units,
                                                                    const Work* __restrict__ work, int n_work,
                                                                    unsigned* counter, int max_wd, int cap, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AdjBuffers b = adj_buffers(smem_raw, max_wd, cap);
    for (;;) {
        // the previous tile's last barrier orders its reads of `w` before this write
        if (threadIdx.x == 0) b.sh->w = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int wi = b.sh->w;
        if (wi >= n_work) return;
        const Work w = work[wi];
        const Unit& u = units[w.unit];
        if (u.fan)
            plan_adjoint_tile<T, KW, true>(u, w.tile, b, Epilogue{1.0f, nullptr, 0.0f, nullptr}, err);
        else if (u.cand3)
            plan_adjoint_tile_parallel<T, KW, 3>(u, w.tile, b, Epilogue{1.0f, nullptr, 0.0f, nullptr}, err);
        else
            plan_adjoint_tile_parallel<T, KW, 0>(u, w.tile, b, Epilogue{1.0f, nullptr, 0.0f, nullptr}, err);
    }
}

// Single image (a batch-1 call): one CTA per tile, the unit passed by value.  NC < 0: fan beam.
template <typename T, int KW, int NC>
__global__ void __launch_bounds__(kPlanThreads) single_adjoint_kernel(const Unit u, const Epilogue ep, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (NC < 0)
        plan_adjoint_tile<T, KW, true>(u, (int)blockIdx.x, adj_buffers(smem_raw, u.wd, u.cfg), ep, err);
    else
        plan_adjoint_tile_parallel<T, KW, NC>(u, (int)blockIdx.x, adj_buffers(smem_raw, u.wd, u.cfg), ep, err);
}

size_t adj_smem_bytes(int max_wd, int cap) {
    return (sizeof(AdjShared) + 15) / 16 * 16 + (size_t)cap * max_wd * (16 + 4 + 4);
}

// Views per chunk at most for windows of max_wd rays: 32 where the staging fits one CTA's shared
// memory, else 16; 0 if not even 16 fit.
int adj_chunk_cap(int max_wd) {
    if (adj_smem_bytes(max_wd, kMaxChunkViews) <= 227 * 1024) return kMaxChunkViews;
    if (adj_smem_bytes(max_wd, 16) <= 227 * 1024) return 16;
    return 0;
}

// --------------------------------------------------------------------------------------- plan

size_t texel_bytes(radon_dtype dt) { return dt == RADON_F32 ? 16 : 8; }

// One image through the plan's kernels, without a plan: the unit is a kernel argument and every
// work item is its own CTA, so a call allocates nothing and can be captured.
constexpr int kSingleForwardViews = 8;    // views per ray block (the plan's default)
constexpr int kSingleForwardLanes = 4;    // lanes per ray: one image's rays alone do not fill the GPU
constexpr int kSingleAdjointViews = 32;   // views per staged chunk (the autotuner's pick at every size)

// Parallel beam: whether every pixel's candidate window holds at most three rays, from the same
// FP32 half width r = (|ax| + |ay|) / b0 + 0.01 the kernel computes (a window shorter than 3
// holds at most 3 integers; 1.49 leaves room for its rounding), and the staged window at least 3.
int three_candidates(const radon_geometry* g) {
    if (g->fan || g->bwd_window + 2 < 3) return 0;
    for (const ViewF& v : g->h_view) {
        const float r = (std::fabs(v.ax) + std::fabs(v.ay)) / v.b0 + 0.01f;
        if (!(r < 1.49f)) return 0;
    }
    return 1;
}

// ---- staged forward: view groups, band bounds, ring shape

constexpr uint32_t kSfSpinLimit = 1u << 22;   // bounded mbarrier polls (~seconds) before giving up

int group_index(int G) { return G >= 8 ? 3 : G >= 4 ? 2 : G >= 2 ? 1 : 0; }

// The unit's view groups for G views per work item (groups of one orientation class).
void set_groups(Unit& u, const radon_geometry* g, int G) {
    const int gi = group_index(G);
    u.groups = g->d_groups + g->group_offset[gi];
    u.n_groups = g->group_count[gi];
}

// Upper bound of the staged forward's band width (texel columns) over every work item and slab of
// geometry g with G views x Dt detectors per item and R rows per slab.  Within one slab's rows
// [y0, y1] the band spans max_l x_l - min_l x_l over the item's extreme-ray lines l; the spread
// max_l x_l(y) - min_l x_l(y) is convex in y, so it is largest at the first or last row any slab
// reaches, and moving within the slab adds at most max |slope| (y1 - y0).  Adds the kernel's margins
// (2 columns each side, floor / ceil, alignment) and slack for its FP32 line evaluation; lines that
// run nearly along the rows count as the whole support.  Cached per geometry and shape.
int staged_band_bound(const radon_geometry* gc, int G, int Dt, int R) {
    radon_geometry* g = const_cast<radon_geometry*>(gc);   // the cache is guarded by band_mu
    const long long key = (1LL << 62) | ((long long)G << 40) | ((long long)Dt << 20) | (long long)R;
    std::lock_guard<std::mutex> lock(g->band_mu);
    auto it = g->band_width.find(key);
    if (it != g->band_width.end()) return it->second;
    const int gi = group_index(G);
    const int n_slabs = (g->n + 3 + R - 1) / R;
    const double y_top = -3.0, y_bot = -2.0 + (double)n_slabs * R + 1.0;
    const int n_dr = (g->D + Dt - 1) / Dt;
    const double cap = g->n + 14.0;
    double maxw = 0.0;
    for (int q = 0; q < g->group_count[gi] && maxw < cap; ++q) {
        const Int2 grp = g->h_groups[g->group_offset[gi] + q];
        const int v0 = grp.x, cnt = grp.y & 0xffff, cls = grp.y >> 16;
        for (int dr = 0; dr < n_dr && maxw < cap; ++dr) {
            const int d0 = dr * Dt, d1 = std::min(d0 + Dt - 1, g->D - 1);
            double lo_t = 1e300, hi_t = -1e300, lo_b = 1e300, hi_b = -1e300, maxsl = 0.0;
            bool flat = false;
            for (int vl = 0; vl < cnt && !flat; ++vl) {
                for (int e = 0; e < 2; ++e) {
                    const RayT& r = g->h_ray[(size_t)(v0 + vl) * g->D + (e ? d1 : d0)];
                    const double X0 = cls ? (double)r.I0 + r.fy0 : (double)r.J0 + r.fx0;
                    const double Y0 = cls ? (double)r.J0 + r.fx0 : (double)r.I0 + r.fy0;
                    const double dX = cls ? (double)r.dyh + r.dyl : (double)r.dxh + r.dxl;
                    const double dY = cls ? (double)r.dxh + r.dxl : (double)r.dyh + r.dyl;
                    if (std::fabs(dY) <= 1e-4 * std::fabs(dX)) {
                        flat = true;
                        break;
                    }
                    const double sl = dX / dY;
                    const double xt = X0 + (y_top - Y0) * sl, xb = X0 + (y_bot - Y0) * sl;
                    lo_t = std::min(lo_t, xt);
                    hi_t = std::max(hi_t, xt);
                    lo_b = std::min(lo_b, xb);
                    hi_b = std::max(hi_b, xb);
                    maxsl = std::max(maxsl, std::fabs(sl));
                }
            }
            const double w = flat ? cap : std::max(hi_t - lo_t, hi_b - lo_b) + maxsl * (R + 2) + 12.0;
            maxw = std::max(maxw, std::min(w, cap));
        }
    }
    int w = (int)std::ceil(maxw);
    w += w & 1;   // even: whole 16-byte blocks of 8-byte texels
    g->band_width[key] = w;
    return w;
}

// Ring of the staged forward for bands of `wbox` texels and `rmax` rows: the most stages (2..4)
// that keep 3 CTAs per SM, else 2 CTAs, else 1; ok = false when not even 2 stages fit one CTA.
struct StagedRing {
    bool ok;
    int stages;
    size_t smem;
};

StagedRing staged_ring(int wbox, int rmax, int qb) {
    constexpr size_t kSmPool = 228 * 1024, kPerCta = 1024, kCtaMax = 227 * 1024;
    for (int ctas : {3, 2, 1})
        for (int st = kSfMaxStages; st >= 2; --st) {
            const size_t smem = sf_smem_bytes(rmax, wbox, qb, st);
            if (smem <= kCtaMax && (size_t)ctas * (smem + kPerCta) <= kSmPool) return StagedRing{true, st, smem};
        }
    return StagedRing{false, 0, 0};
}

// Raises kernel K's dynamic shared memory limit on the current device to `smem`, never lowering it:
// plans of different shapes and the batch-1 calls share the kernels, and a launch needs the limit at
// least as large as its own request.  Not thread-safe, like the other attribute caches here.
template <auto K>
cudaError_t raise_smem_attr(size_t smem) {
    static size_t attr_bytes[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t& cur = attr_bytes[dev & 63];
    if (smem <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

template <typename T>
cudaError_t staged_smem_attr(size_t smem) {
    return raise_smem_attr<staged_forward_kernel<T>>(smem);
}

Unit single_unit(const radon_geometry* g, const void* in, void* out, int cfg) {
    Unit u;
    u.in = in;
    u.out = out;
    u.rays = g->d_ray;
    u.nks = g->d_nk;
    u.views = g->d_view;
    u.q_off = 0;
    u.n = g->n;
    u.V = g->V;
    u.D = g->D;
    u.h = (float)g->h;
    u.ih2 = (float)(1.0 / (g->h * g->h));
    u.wd = g->bwd_window + 2;
    u.cfg = cfg;
    u.lanes = kSingleForwardLanes;
    u.fan = g->fan;
    u.cand3 = three_candidates(g);
    u.R = 0;
    u.staged = 0;
    set_groups(u, g, cfg);
    return u;
}

template <typename T>
radon_status single_forward_t(const radon_geometry* g, const void* img, void* sino, void* ws, const Epilogue& ep,
                              cudaStream_t s) {
    using Q = typename Quad<T>::type;
    const Unit u = single_unit(g, img, sino, kSingleForwardViews);
    const long long texels = 2 * sq_frame(g->n);
    const unsigned pack_blocks = (unsigned)std::min<long long>((texels + 255) / 256, 152LL * 64);
    sq_pack_single_kernel<T><<<pack_blocks, 256, 0, s>>>(static_cast<const T*>(img), g->n, static_cast<Q*>(ws));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "single-image pack launch");
    count_launches(1);
    // every sample one texel load through L1, four lanes per ray: a single image's rays alone fill
    // the GPU only thinly, and the staged kernel measured slower here (512^2, 60 views: 0.39 vs 0.09 ms)
    const int Dl = kPlanThreads / (kSingleForwardLanes * kSingleForwardViews);
    const long long blocks = (long long)((g->V + kSingleForwardViews - 1) / kSingleForwardViews) * ((g->D + Dl - 1) / Dl);
    single_forward_kernel<T><<<(unsigned)blocks, kPlanThreads, 0, s>>>(u, static_cast<const Q*>(ws), ep);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "single-image forward launch");
    count_launches(1);
    return RADON_OK;
}

template <typename T, int KW, int NC>
radon_status single_backward_tk(const Unit& u, long long tiles, size_t smem, const Epilogue& ep, int* err,
                                cudaStream_t s) {
    auto kern = single_adjoint_kernel<T, KW, NC>;
    const cudaError_t ea = raise_smem_attr<single_adjoint_kernel<T, KW, NC>>(smem);
    if (ea != cudaSuccess) return cuda_fail(ea, "single-image adjoint shared memory");
    kern<<<(unsigned)tiles, kPlanThreads, smem, s>>>(u, ep, err);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "single-image adjoint launch");
    count_launches(1);
    return RADON_OK;
}

template <typename T>
radon_status single_backward_t(const radon_geometry* g, const void* sino, void* img, const Epilogue& ep, cudaStream_t s,
                               std::string* why) {
    const int kw_needed = (int)std::floor(2.0 * std::sqrt(2.0) / g->h + 2e-4) + 1;
    if (kw_needed > 6) {
        *why = "sampling step too small for the single-image adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const int cap = adj_chunk_cap(g->bwd_window + 2);
    if (cap == 0) {
        *why = "detector window too wide for the single-image adjoint";
        return RADON_ERR_UNSUPPORTED;
    }
    const Unit u = single_unit(g, sino, img, std::min(kSingleAdjointViews, cap));
    const size_t smem = adj_smem_bytes(u.wd, u.cfg);
    int* err = device_error_word();
    if (err == nullptr) {
        *why = "device error word unavailable";
        return RADON_ERR_CUDA;
    }
    const long long tiles_x = (g->n + kBwdTile - 1) / kBwdTile;
    const long long tiles = tiles_x * tiles_x;
    if (g->fan)
        return kw_needed <= 3 ? single_backward_tk<T, 3, -1>(u, tiles, smem, ep, err, s)
                              : single_backward_tk<T, 6, -1>(u, tiles, smem, ep, err, s);
    if (u.cand3)
        return kw_needed <= 3 ? single_backward_tk<T, 3, 3>(u, tiles, smem, ep, err, s)
                              : single_backward_tk<T, 6, 3>(u, tiles, smem, ep, err, s);
    return kw_needed <= 3 ? single_backward_tk<T, 3, 0>(u, tiles, smem, ep, err, s)
                          : single_backward_tk<T, 6, 0>(u, tiles, smem, ep, err, s);
}

}  // namespace

size_t single_forward_workspace_bytes(const radon_geometry* g, radon_dtype dt) {
    return 2 * (size_t)sq_frame(g->n) * texel_bytes(dt);
}

radon_status launch_forward_single(const radon_geometry* g, const void* img, void* sino, radon_dtype dt, void* ws,
                                   const Epilogue& ep, cudaStream_t s) {
    switch (dt) {
        case RADON_F16: return single_forward_t<__half>(g, img, sino, ws, ep, s);
        case RADON_BF16: return single_forward_t<__nv_bfloat16>(g, img, sino, ws, ep, s);
        default: return single_forward_t<float>(g, img, sino, ws, ep, s);
    }
}

radon_status launch_backward_single(const radon_geometry* g, const void* sino, void* img, radon_dtype dt,
                                    const Epilogue& ep, cudaStream_t s, std::string* why) {
    switch (dt) {
        case RADON_F16: return single_backward_t<__half>(g, sino, img, ep, s, why);
        case RADON_BF16: return single_backward_t<__nv_bfloat16>(g, sino, img, ep, s, why);
        default: return single_backward_t<float>(g, sino, img, ep, s, why);
    }
}

}  // namespace radon

using namespace radon;

struct radon_plan {
    uint64_t magic = kPlanMagic;
    int direction = 0;
    radon_dtype dtype = RADON_F32;
    int device = 0;
    int kw = 3;
    int max_wd = 0;
    int cap = kMaxChunkViews;   // adjoint: views per chunk at most (its shared memory holds that many)
    int ctas = 0;
    size_t smem = 0;
    std::vector<Unit> units;
    std::vector<int> unit_item;
    std::vector<int> item_cfg;
    std::vector<int> item_lanes;
    std::vector<int> item_rows;
    std::vector<const radon_geometry*> unit_geom;
    bool staged_ok = false;     // forward: the staged kernel may serve units (its ring fits)
    int wbox = 0, rmax = 0, stages = 0, ctas_staged = 0;
    int n_work_staged = 0;      // forward: the work list's first n_work_staged items run the staged kernel
    std::vector<Work> work;
    std::vector<long long> prefix;   // forward: texel offsets, n_units + 1
    Unit* d_units = nullptr;
    Work* d_work = nullptr;
    long long* d_prefix = nullptr;
    unsigned* d_counter = nullptr;
    void* d_quads = nullptr;
    long long total_texels = 0;
};

namespace radon {

namespace {

void free_plan(radon_plan* p) {
    if (p == nullptr) return;
    cudaFree(p->d_units);
    cudaFree(p->d_work);
    cudaFree(p->d_prefix);
    cudaFree(p->d_counter);
    cudaFree(p->d_quads);
    p->magic = 0;
    delete p;
}

// Work list over the units in `sel`, largest work items first: the staged kernel's units first (their
// count in *n_staged), then the others.
std::vector<Work> build_work(const radon_plan* p, const std::vector<int>& sel, int* n_staged) {
    std::vector<int> order(sel);
    auto cost = [&](int ui) -> double {
        const Unit& u = p->units[ui];
        return p->direction == 0 ? (double)u.n : (double)u.V;   // per work item
    };
    auto staged = [&](int ui) { return p->direction == 0 && p->units[ui].staged != 0; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (staged(a) != staged(b)) return staged(a);
        return cost(a) > cost(b);
    });
    std::vector<Work> w;
    *n_staged = 0;
    for (int ui : order) {
        const Unit& u = p->units[ui];
        int tiles;
        if (staged(ui)) {
            const int Dt = kSfConsumers / (u.lanes * u.cfg);
            tiles = u.n_groups * ((u.D + Dt - 1) / Dt);
            *n_staged += tiles;
        } else if (p->direction == 0) {
            const int G = u.cfg, Dt = kPlanThreads / (u.lanes * G);
            tiles = ((u.V + G - 1) / G) * ((u.D + Dt - 1) / Dt);
        } else {
            const int t = (u.n + kBwdTile - 1) / kBwdTile;
            tiles = t * t;
        }
        for (int t = 0; t < tiles; ++t) w.push_back(Work{ui, t});
    }
    return w;
}

radon_status upload_work(const std::vector<Work>& w, Work** dst) {
    cudaFree(*dst);
    *dst = nullptr;
    if (w.empty()) return RADON_OK;
    cudaError_t e = cudaMalloc(dst, w.size() * sizeof(Work));
    if (e != cudaSuccess) return fail(RADON_ERR_OOM, "cudaMalloc of the work list failed");
    e = cudaMemcpy(*dst, w.data(), w.size() * sizeof(Work), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "work list upload");
    return RADON_OK;
}

radon_status upload_units(radon_plan* p) {
    cudaError_t e = cudaMemcpy(p->d_units, p->units.data(), p->units.size() * sizeof(Unit), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "unit table upload");
    return RADON_OK;
}

template <typename T>
// Runs the plan over the work list d_work (n_work items, the first n_staged of them staged-kernel
// items): forward = pack, then the staged kernel and the L1 gather, each persistent over its items
// with its own counter; adjoint = one persistent kernel.
radon_status launch_t(const radon_plan* p, const Work* d_work, int n_work, int n_staged, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p->d_counter, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "work counter reset");
    if (n_work == 0) return RADON_OK;
    using Q = typename Quad<T>::type;
    if (p->direction == 0) {
        const unsigned blocks = (unsigned)std::min<long long>((p->total_texels + 255) / 256, 152LL * 64);
        sq_pack_kernel<T><<<blocks, 256, 0, s>>>(p->d_units, p->d_prefix, (int)p->units.size(), p->total_texels,
                                                 static_cast<Q*>(p->d_quads));
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "plan pack launch");
        if (n_staged > 0) {
            int* err = device_error_word();
            if (err == nullptr) return fail(RADON_ERR_CUDA, "device error word unavailable");
            const SfArgs a{p->d_units, d_work, n_staged, p->d_counter, p->d_quads, p->wbox,
                           sf_pitch(p->wbox, (int)sizeof(Q)), p->rmax, p->stages, err, kSfSpinLimit, identity_epilogue()};
            staged_forward_kernel<T><<<p->ctas_staged, kSfThreads, p->smem, s>>>(a);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "plan staged forward launch");
            count_launches(1);
        }
        if (n_work > n_staged)
            plan_forward_kernel<T><<<p->ctas, kPlanThreads, 0, s>>>(p->d_units, d_work + n_staged, n_work - n_staged,
                                                                   p->d_counter + 1, static_cast<const Q*>(p->d_quads));
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "plan forward launch");
        count_launches(n_work > n_staged ? 2 : 1);
    } else {
        int* err = device_error_word();
        if (err == nullptr) return fail(RADON_ERR_CUDA, "device error word unavailable");
        if (p->kw == 3)
            plan_adjoint_kernel<T, 3><<<p->ctas, kPlanThreads, p->smem, s>>>(p->d_units, d_work, n_work, p->d_counter,
                                                                            p->max_wd, p->cap, err);
        else
            plan_adjoint_kernel<T, 6><<<p->ctas, kPlanThreads, p->smem, s>>>(p->d_units, d_work, n_work, p->d_counter,
                                                                            p->max_wd, p->cap, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "plan adjoint launch");
        count_launches(1);
    }
    return RADON_OK;
}

radon_status launch_plan(const radon_plan* p, const Work* d_work, int n_work, int n_staged, cudaStream_t s) {
    switch (p->dtype) {
        case RADON_F16: return launch_t<__half>(p, d_work, n_work, n_staged, s);
        case RADON_BF16: return launch_t<__nv_bfloat16>(p, d_work, n_work, n_staged, s);
        default: return launch_t<float>(p, d_work, n_work, n_staged, s);
    }
}

template <typename T>
radon_status occupancy_t(radon_plan* p) {
    int per_sm = 0;
    cudaError_t e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (p->direction == 0 && p->staged_ok && p->smem > 0) {   // the staged kernel at the current ring
        int per_sm_s = 0;
        e = staged_smem_attr<T>(p->smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, staged_forward_kernel<T>, kSfThreads, p->smem);
        if (e != cudaSuccess) return cuda_fail(e, "plan occupancy query");
        p->ctas_staged = std::max(1, per_sm_s) * sms;
    }
    if (p->direction == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_forward_kernel<T>, kPlanThreads, 0);
    } else if (p->kw == 3) {
        e = raise_smem_attr<plan_adjoint_kernel<T, 3>>(p->smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_adjoint_kernel<T, 3>, kPlanThreads, p->smem);
    } else {
        e = raise_smem_attr<plan_adjoint_kernel<T, 6>>(p->smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_adjoint_kernel<T, 6>, kPlanThreads, p->smem);
    }
    if (e != cudaSuccess) return cuda_fail(e, "plan occupancy query");
    p->ctas = std::max(1, per_sm) * sms;
    return RADON_OK;
}

radon_status occupancy(radon_plan* p) {
    switch (p->dtype) {
        case RADON_F16: return occupancy_t<__half>(p);
        case RADON_BF16: return occupancy_t<__nv_bfloat16>(p);
        default: return occupancy_t<float>(p);
    }
}

// A tuned shape: views per forward work item or adjoint chunk, lanes per forward ray, texel rows per
// staged forward slab (0 for the L1 gather and the adjoint; rows > 0 selects the staged kernel).
struct Shape {
    int views, lanes, rows;
    bool operator==(const Shape& o) const { return views == o.views && lanes == o.lanes && rows == o.rows; }
};

// Tuning cache: when RADON_TUNE_CACHE names a file, every tuned group's pick is appended to it as
// one line "<key> <views> <lanes> <rows>" and later plans take a group's pick from the file (the last
// line of a key wins) instead of timing its candidates.  The key is the direction, storage type,
// image size, geometry kind and forward kernel -- the group the tuner times together.
using TuneCache = std::map<std::string, Shape>;

std::string tune_key(int direction, radon_dtype dt, int n, int fan, int kernels) {
    static const char* const names[3] = {"_gather", "_any", "_staged"};
    return "plan" + std::to_string(direction) + "_dt" + std::to_string((int)dt) + "_n" + std::to_string(n) +
           (fan ? "_fan" : "_par") + (direction == 0 ? names[kernels + 1] : "");
}

TuneCache load_tune_cache() {
    TuneCache c;
    const char* path = std::getenv("RADON_TUNE_CACHE");
    if (path == nullptr || path[0] == 0) return c;
    std::FILE* f = std::fopen(path, "r");
    if (f == nullptr) return c;
    char key[128];
    int v = 0, l = 0, r = 0;
    while (std::fscanf(f, "%127s %d %d %d", key, &v, &l, &r) == 4) c[key] = Shape{v, l, r};
    std::fclose(f);
    return c;
}

void store_tune_cache(const std::string& key, const Shape& pick) {
    const char* path = std::getenv("RADON_TUNE_CACHE");
    if (path == nullptr || path[0] == 0) return;
    std::FILE* f = std::fopen(path, "a");   // one short line per append
    if (f == nullptr) return;
    std::fprintf(f, "%s %d %d %d\n", key.c_str(), pick.views, pick.lanes, pick.rows);
    std::fclose(f);
}

constexpr int kPlanForwardRows = 16;   // texel rows per staged slab by default

// Forward shape of unit k (views per work item, lanes per ray; rows per slab > 0 = the staged kernel)
// and its view groups.
void set_forward_shape(radon_plan* p, int k, const Shape& sh) {
    Unit& u = p->units[k];
    u.cfg = sh.views;
    u.lanes = sh.lanes;
    u.staged = sh.rows > 0 ? 1 : 0;
    u.R = sh.rows > 0 ? sh.rows : kPlanForwardRows;
    set_groups(u, p->unit_geom[k], u.cfg);
}

// Staged forward over units `sel`: widest band, most rows and the ring they need (the plan's launch
// shape); false when the ring does not fit one CTA's shared memory.
bool staged_fit(radon_plan* p, const std::vector<int>& sel) {
    int wbox = 2, rmax = 1;
    for (int k : sel) {
        const Unit& u = p->units[k];
        if (!u.staged) continue;
        const int Dt = kSfConsumers / (u.lanes * u.cfg);
        wbox = std::max(wbox, staged_band_bound(p->unit_geom[k], u.cfg, Dt, u.R));
        rmax = std::max(rmax, u.R);
    }
    const StagedRing ring = staged_ring(wbox, rmax, (int)texel_bytes(p->dtype));
    if (!ring.ok) return false;
    p->wbox = wbox;
    p->rmax = rmax;
    p->stages = ring.stages;
    p->smem = ring.smem;
    return true;
}

// Times `reps` launches of the plan restricted to units `sel`; returns the median in ms (3e38 for a
// staged shape whose ring does not fit).
radon_status time_subset(radon_plan* p, const std::vector<int>& sel, float* ms) {
    if (p->direction == 0 && p->staged_ok) {
        if (!staged_fit(p, sel)) {
            *ms = 3.0e38f;
            return RADON_OK;
        }
        const radon_status so = occupancy(p);
        if (so != RADON_OK) return so;
    }
    int n_staged = 0;
    const std::vector<Work> w = build_work(p, sel, &n_staged);
    Work* d = nullptr;
    radon_status st = upload_work(w, &d);
    if (st != RADON_OK) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int r = 0; r < 4 && st == RADON_OK; ++r) {
        cudaEventRecord(e0, 0);
        st = launch_plan(p, d, (int)w.size(), n_staged, 0);
        cudaEventRecord(e1, 0);
        if (st == RADON_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float x = 0.f;
            cudaEventElapsedTime(&x, e0, e1);
            if (r > 0) t.push_back(x);   // the first run warms up
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (st != RADON_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "autotune run");
    std::sort(t.begin(), t.end());
    *ms = t.empty() ? 0.f : t[t.size() / 2];
    return RADON_OK;
}

}  // namespace

}  // namespace radon

extern "C" RADON_API radon_status radon_batch_plan_create(const radon_item* items, int n, int direction,
                                                          radon_dtype dtype, const radon_plan_options* options,
                                                          radon_plan** out) {
    if (out == nullptr) return fail(RADON_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && items == nullptr)) return fail(RADON_ERR_INVALID_ARG, "items is NULL or n < 0");
    if (direction != 0 && direction != 1) return fail(RADON_ERR_INVALID_ARG, "direction must be 0 (forward) or 1 (adjoint)");
    if (dtype != RADON_F32 && dtype != RADON_F16 && dtype != RADON_BF16)
        return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    const int fv = options ? options->forward_views : 0, av = options ? options->adjoint_views : 0;
    const int fl = options ? options->forward_lanes : 0;
    const int fr = options ? options->forward_rows : 0;
    const int fk = options ? options->forward_kernel : 0;
    if (fv < 0 || (fv > 0 && fv != 1 && fv != 2 && fv != 4 && fv != 8))
        return fail(RADON_ERR_INVALID_ARG, "forward_views must be 0, 1, 2, 4 or 8");
    if (fl != 0 && fl != 1 && fl != kPlanMaxLanes) return fail(RADON_ERR_INVALID_ARG, "forward_lanes must be 0, 1 or 4");
    if (fr != 0 && fr != 8 && fr != 16 && fr != 32) return fail(RADON_ERR_INVALID_ARG, "forward_rows must be 0, 8, 16 or 32");
    if (fk < -1 || fk > 1) return fail(RADON_ERR_INVALID_ARG, "forward_kernel must be -1, 0 or 1");
    if (av < 0 || (av > 0 && av != 4 && av != 8 && av != 16 && av != 32))
        return fail(RADON_ERR_INVALID_ARG, "adjoint_views must be 0, 4, 8, 16 or 32");
    const bool autotune = options == nullptr || options->autotune != 0;
    const size_t es = dtype == RADON_F32 ? 4 : 2;
    for (int i = 0; i < n; ++i) {
        const radon_item& it = items[i];
        const radon_geometry* g = it.geometry;
        if (g == nullptr || g->magic != kGeometryMagic)
            return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": geometry is not a live geometry");
        if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": host-only geometry");
        if (it.batch < 0) return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": batch < 0");
        if (it.batch > 0 && (it.in == nullptr || it.out == nullptr))
            return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": NULL buffer");
        if (it.batch > 0 && (((uintptr_t)it.in % es) != 0 || ((uintptr_t)it.out % es) != 0))
            return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": buffer not aligned to its element size");
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    for (int i = 0; i < n; ++i)
        if (items[i].geometry->device != dev)
            return fail(RADON_ERR_INVALID_ARG, "item " + std::to_string(i) + ": geometry on another device");
    radon_plan* p = new (std::nothrow) radon_plan();
    if (p == nullptr) return fail(RADON_ERR_OOM, "host allocation failed");
    p->direction = direction;
    p->dtype = dtype;
    p->device = dev;
    p->item_cfg.assign(n, 0);
    p->item_lanes.assign(n, 0);
    p->item_rows.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const radon_item& it = items[i];
        const radon_geometry* g = it.geometry;
        const long long in_sz = direction == 0 ? (long long)g->n * g->n : (long long)g->V * g->D;
        const long long out_sz = direction == 0 ? (long long)g->V * g->D : (long long)g->n * g->n;
        for (int b = 0; b < it.batch; ++b) {
            Unit u;
            u.in = static_cast<const unsigned char*>(it.in) + (size_t)b * in_sz * es;
            u.out = static_cast<unsigned char*>(it.out) + (size_t)b * out_sz * es;
            u.rays = g->d_ray;
            u.nks = g->d_nk;
            u.views = g->d_view;
            u.q_off = 0;
            u.n = g->n;
            u.V = g->V;
            u.D = g->D;
            u.h = (float)g->h;
            u.ih2 = (float)(1.0 / (g->h * g->h));
            u.wd = g->bwd_window + 2;
            u.fan = g->fan;
            u.cand3 = direction == 1 ? three_candidates(g) : 0;
            u.cfg = direction == 0 ? (fv > 0 ? fv : 8) : (av > 0 ? av : kMaxChunkViews);
            u.lanes = direction == 0 && fl > 0 ? fl : 1;
            u.R = fr > 0 ? fr : kPlanForwardRows;
            // the kernel before tuning: staged when asked for (or rows given), else the L1 gather
            u.staged = direction == 0 && (fk == 1 || (fk == 0 && fr > 0)) ? 1 : 0;
            set_groups(u, g, u.cfg);
            p->units.push_back(u);
            p->unit_item.push_back(i);
            p->unit_geom.push_back(g);
            p->max_wd = std::max(p->max_wd, u.wd);
            if (direction == 1) {
                // samples per candidate window: the window spans 2 (|dx|+|dy|)/h^2 <= 2 sqrt(2) / h
                const int kw_needed = (int)std::floor(2.0 * std::sqrt(2.0) / g->h + 2e-4) + 1;
                if (kw_needed > 6) {
                    free_plan(p);
                    return fail(RADON_ERR_UNSUPPORTED, "item " + std::to_string(i) +
                                                           ": sampling step too small for the adjoint plan");
                }
                if (kw_needed > 3) p->kw = 6;
            }
        }
    }
    radon_status st = RADON_OK;
    const size_t nu = p->units.size();
    if (direction == 0) {
        p->prefix.assign(nu + 1, 0);
        for (size_t k = 0; k < nu; ++k) {
            p->units[k].q_off = p->prefix[k];
            p->prefix[k + 1] = p->prefix[k] + 2 * sq_frame(p->units[k].n);
        }
        p->total_texels = p->prefix[nu];
        // the staged kernel may serve units unless refused; its ring must fit the units that start on it
        std::vector<int> all(nu);
        for (size_t k = 0; k < nu; ++k) all[k] = (int)k;
        p->staged_ok = fk >= 0;
        if (p->staged_ok && nu > 0 && !staged_fit(p, all)) {
            if (fk == 1 || fr > 0) {
                free_plan(p);
                return fail(RADON_ERR_UNSUPPORTED, "the staged forward's bands do not fit shared memory");
            }
            p->staged_ok = false;
        }
    } else {
        p->cap = adj_chunk_cap(std::max(p->max_wd, 1));
        if (p->cap == 0) {
            free_plan(p);
            return fail(RADON_ERR_UNSUPPORTED, "detector window too wide for the adjoint plan's shared memory");
        }
        if (av > p->cap) {
            free_plan(p);
            return fail(RADON_ERR_UNSUPPORTED, "adjoint_views " + std::to_string(av) +
                                                   " exceeds the shared memory of these detector windows");
        }
        p->smem = adj_smem_bytes(std::max(p->max_wd, 1), p->cap);
        for (Unit& u : p->units) u.cfg = std::min(u.cfg, p->cap);   // the default chunk where it fits
    }
    if (nu > 0) {
        if (cudaMalloc(&p->d_units, nu * sizeof(Unit)) != cudaSuccess ||
            cudaMalloc(&p->d_counter, 2 * sizeof(unsigned)) != cudaSuccess ||
            (direction == 0 && (cudaMalloc(&p->d_prefix, (nu + 1) * sizeof(long long)) != cudaSuccess ||
                                cudaMalloc(&p->d_quads, (size_t)p->total_texels * texel_bytes(dtype)) != cudaSuccess))) {
            cudaGetLastError();
            free_plan(p);
            return fail(RADON_ERR_OOM, "device allocation for the plan failed");
        }
        if (direction == 0) {
            e = cudaMemcpy(p->d_prefix, p->prefix.data(), (nu + 1) * sizeof(long long), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                free_plan(p);
                return cuda_fail(e, "plan upload");
            }
        }
        st = occupancy(p);
        if (st == RADON_OK) st = upload_units(p);
        // Autotuner: per image size (and geometry kind), time each candidate shape on that group's
        // units alone -- forward: views per work item x lanes per ray (x texel rows per slab for the
        // staged kernel), adjoint: views per chunk -- unless the options fix it; a tuning cache
        // (RADON_TUNE_CACHE) answers groups tuned before.
        const bool fixed = direction == 0 ? (fv > 0 && fl > 0 && (fk != 1 || fr > 0)) : av > 0;
        if (st == RADON_OK && autotune && !fixed) {
            std::vector<Shape> cand;
            if (direction == 0) {
                // the L1 gather: views per ray block x lanes per ray
                if (fk <= 0 && fr == 0)
                    for (int G : {8, 4, 2, 1})
                        for (int lanes : {1, kPlanMaxLanes})
                            if ((fv == 0 || G == fv) && (fl == 0 || lanes == fl)) cand.push_back(Shape{G, lanes, 0});
                // the staged kernel: views per item x rows per slab (one lane per ray unless asked: four
                // lanes measured slower at every size)
                if (p->staged_ok)
                    for (int G : {8, 4, 2})
                        for (int R : {16, 32})
                            if ((fv == 0 || G == fv) && (fr == 0 || R == fr))
                                cand.push_back(Shape{G, fl > 0 ? fl : 1, R});
            } else {
                for (int cv : {4, 8, 16, 32})
                    if (cv <= p->cap) cand.push_back(Shape{cv, 1, 0});
            }
            std::map<std::pair<int, int>, std::vector<int>> groups;   // (n, fan) -> units
            for (size_t k = 0; k < nu; ++k) groups[{p->units[k].n, p->units[k].fan}].push_back((int)k);
            const TuneCache cache = load_tune_cache();
            auto apply = [&](const std::vector<int>& ks, const Shape& sh) {
                for (int k : ks) {
                    if (direction == 0) set_forward_shape(p, k, sh);
                    else p->units[k].cfg = sh.views;
                }
            };
            for (auto& kv : groups) {
                const std::string key = tune_key(direction, dtype, kv.first.first, kv.first.second, fk);
                auto hit = cache.find(key);
                Shape best_c = cand[0];
                if (hit != cache.end() && std::find(cand.begin(), cand.end(), hit->second) != cand.end()) {
                    best_c = hit->second;
                } else {
                    float best = 3.0e38f;
                    for (size_t c = 0; c < cand.size() && st == RADON_OK; ++c) {
                        apply(kv.second, cand[c]);
                        st = upload_units(p);
                        float ms = 0.f;
                        if (st == RADON_OK) st = time_subset(p, kv.second, &ms);
                        if (st == RADON_OK && ms < best) {
                            best = ms;
                            best_c = cand[c];
                        }
                    }
                    if (st == RADON_OK) store_tune_cache(key, best_c);
                }
                apply(kv.second, best_c);
            }
            if (st == RADON_OK) st = upload_units(p);
        }
        if (st == RADON_OK && direction == 0 && p->staged_ok) {   // the staged launch of the whole plan
            std::vector<int> all(nu);
            for (size_t k = 0; k < nu; ++k) all[k] = (int)k;
            if (!staged_fit(p, all)) {
                // the size groups' picks together need more shared memory than one CTA has: the staged
                // units fall back to the gather's default shape, unless the staged kernel was required
                if (fk == 1) {
                    st = fail(RADON_ERR_UNSUPPORTED, "the staged forward's bands do not fit shared memory");
                } else {
                    for (size_t k = 0; k < nu; ++k)
                        if (p->units[k].staged) set_forward_shape(p, (int)k, Shape{8, 1, 0});
                    st = upload_units(p);
                }
            }
            if (st == RADON_OK) st = occupancy(p);
        }
    }
    if (st == RADON_OK) {
        std::vector<int> all(nu);
        for (size_t k = 0; k < nu; ++k) all[k] = (int)k;
        p->work = build_work(p, all, &p->n_work_staged);
        st = upload_work(p->work, &p->d_work);
    }
    if (st != RADON_OK) {
        free_plan(p);
        return st;
    }
    for (size_t k = 0; k < nu; ++k) {
        p->item_cfg[p->unit_item[k]] = p->units[k].cfg;
        p->item_lanes[p->unit_item[k]] = p->units[k].lanes;
        p->item_rows[p->unit_item[k]] = direction == 0 && p->units[k].staged ? p->units[k].R : 0;
    }
    *out = p;
    return RADON_OK;
}

extern "C" RADON_API radon_status radon_batch_plan_launch(radon_plan* p, void* stream) {
    if (p == nullptr || p->magic != kPlanMagic) return fail(RADON_ERR_INVALID_ARG, "plan is not a live plan");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(RADON_ERR_INVALID_ARG, "plan lives on another device");
    if (p->units.empty()) return RADON_OK;
    return launch_plan(p, p->d_work, (int)p->work.size(), p->n_work_staged, (cudaStream_t)stream);
}

extern "C" RADON_API radon_status radon_batch_plan_get_info(const radon_plan* p, radon_plan_info* info) {
    if (p == nullptr || p->magic != kPlanMagic) return fail(RADON_ERR_INVALID_ARG, "plan is not a live plan");
    if (info == nullptr) return fail(RADON_ERR_INVALID_ARG, "info is NULL");
    info->units = (int)p->units.size();
    info->work_items = (int)p->work.size();
    info->ctas = p->ctas;
    info->direction = p->direction;
    return RADON_OK;
}

extern "C" RADON_API radon_status radon_batch_plan_item_config(const radon_plan* p, int item, int* views) {
    if (p == nullptr || p->magic != kPlanMagic) return fail(RADON_ERR_INVALID_ARG, "plan is not a live plan");
    if (item < 0 || item >= (int)p->item_cfg.size() || views == nullptr)
        return fail(RADON_ERR_INVALID_ARG, "item out of range or views is NULL");
    *views = p->item_cfg[item];
    return RADON_OK;
}

extern "C" RADON_API radon_status radon_batch_plan_item_shape(const radon_plan* p, int item, int* views, int* lanes) {
    if (p == nullptr || p->magic != kPlanMagic) return fail(RADON_ERR_INVALID_ARG, "plan is not a live plan");
    if (item < 0 || item >= (int)p->item_cfg.size() || views == nullptr || lanes == nullptr)
        return fail(RADON_ERR_INVALID_ARG, "item out of range or NULL output");
    *views = p->item_cfg[item];
    *lanes = p->item_lanes[item];
    return RADON_OK;
}

extern "C" RADON_API radon_status radon_batch_plan_item_rows(const radon_plan* p, int item, int* rows) {
    if (p == nullptr || p->magic != kPlanMagic) return fail(RADON_ERR_INVALID_ARG, "plan is not a live plan");
    if (item < 0 || item >= (int)p->item_rows.size() || rows == nullptr)
        return fail(RADON_ERR_INVALID_ARG, "item out of range or rows is NULL");
    *rows = p->item_rows[item];
    return RADON_OK;
}

extern "C" RADON_API void radon_batch_plan_destroy(radon_plan* p) {
    if (p == nullptr || p->magic != kPlanMagic) return;
    free_plan(p);
}
