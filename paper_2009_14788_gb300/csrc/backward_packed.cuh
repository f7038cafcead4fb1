// Packed gather adjoint (the exact transpose of the forward projection, computed pixel by pixel with
// no atomics) and, with KW = 0, the interpolating backprojector.
//
// The sinogram batch is packed once (pack.cu) into rows of BG images per detector,
// [group][view][det][BG] in the storage type (FP32 rows carry four padding words).  One CTA owns a
// 16 x 16 pixel tile of BG images and loops over every view in chunks of kBwdPViews views, through a
// ring of `stages` TMA destinations:
//   * the producer warp computes each view's detector window for the tile (and checks that it holds
//     every pixel's candidate rays), then issues per view one TMA copy of the window's rows
//     [det][BG] and one of the window's rows of the ray table, up to the ring's depth ahead;
//   * the 256 consumer threads (one pixel each), once a chunk has landed, convert 16-bit windows to
//     FP32 rows of pitch (BG + 4) words in a double buffer (FP32 windows land in that layout
//     directly), re-base each landed ray on the tile in place -- reference sample, step and the
//     window constant C of its candidate samples -- meet at a named barrier and gather: each thread
//     owns two vertically neighbouring pixels (one for 32-image groups); for every candidate ray of
//     either pixel, each pixel's KW sample weights once for all BG images, then one FP32 FMA per
//     image and pixel from one row of loads.
// Shared-memory addresses stay 32-bit (explicit ld/st.shared), and no index needs a division.
// The row pitch of (BG + 4) words is an odd number of 16-byte units, so the 16-byte loads of eight
// lanes that read eight consecutive detectors fall in eight different bank groups.
#pragma once

#include <string>

#include "backward_tiled.cuh"
#include "dtype.cuh"
#include "epilogue.cuh"
#include "f32x2.cuh"
#include "radon_internal.h"
#include "tensor_map.h"
#include "tma.cuh"

namespace radon {

constexpr int kBwdPViews = 4;            // views per chunk
constexpr int kBwdPMaxStages = 4;        // ring depth limit (mbarrier slots in the header)
// Pixels per consumer thread: a vertical pair of neighbours shares its candidate rays, so every ray
// record and window row loaded from shared memory serves both pixels' accumulators (16-image groups);
// 32-image groups keep one pixel per thread (their accumulators already fill the registers).
template <int BG>
struct BwdPShape {
    static constexpr int PX = BG <= 16 ? 2 : 1;
    static constexpr int kConsumers = kBwdThreads / PX;
    static constexpr int kThreads = kConsumers + 32;
    static constexpr int kCtasPerSm = PX == 2 ? 4 : 2;   // resident CTAs the launch bounds ask for
};
constexpr size_t kBwdPHeader = 1024;     // barriers, flags, windows and view maps of the ring

template <typename T, int BG>
struct BwdPLayout {
    static constexpr bool kConv = sizeof(T) == 2;              // 16-bit windows are converted in smem
    static constexpr int kRowElems = kConv ? BG : BG + 4;      // elements per detector in the workspace
    static constexpr int kPitch = (BG + 4) * 4;                // bytes per detector of an FP32 window row
    static_assert(((BG + 4) / 4) % 2 == 1, "the FP32 row pitch must be an odd number of 16-byte units");
};

__host__ __device__ inline size_t bwdp_round128(size_t x) { return (x + 127) / 128 * 128; }

// Shared-memory plan of one CTA, identical on host and device.
struct BwdPSmem {
    size_t yst_view;   // TMA'd window rows of one view
    size_t rst_view;   // TMA'd ray rows of one view (re-based in place)
    size_t stage;      // one ring slot (kBwdPViews views)
    size_t yf_view;    // converted FP32 window of one view (16-bit storage only)
    size_t yf_buf;     // one of the two converted buffers
    size_t total;      // dynamic shared memory of the launch (with 128 B of alignment slack)
};

template <typename T, int BG>
__host__ __device__ inline BwdPSmem bwdp_smem(int wd, int stages, bool rays) {
    using L = BwdPLayout<T, BG>;
    BwdPSmem m;
    m.yst_view = bwdp_round128((size_t)wd * L::kRowElems * sizeof(T));
    m.rst_view = rays ? bwdp_round128((size_t)wd * 32) : 0;
    m.stage = (size_t)kBwdPViews * (m.yst_view + m.rst_view);
    m.yf_view = L::kConv ? bwdp_round128((size_t)wd * L::kPitch) : 0;
    m.yf_buf = (size_t)kBwdPViews * m.yf_view;
    m.total = 128 + kBwdPHeader + (size_t)stages * m.stage + 2 * m.yf_buf;
    return m;
}

struct BwdPArgs {
    const ViewF* views;
    void* img;
    int n, V, D, B;
    float h;           // output scale (the step; 1 for the interpolating backprojector)
    float ih2;         // 1 / step^2 (every ray's step has length h)
    int wd;            // detector window per view (rows copied per view)
    int stages;        // ring depth (2..kBwdPMaxStages)
    int tiles_x;
    int out_dtype;     // radon_dtype of the output image
    int* err;
    uint32_t spin_limit;
    Epilogue ep;
    const float4* tab_w;   // weight table (TAB kernels): [tile][view][pair] two float4s, see bwdp_table_kernel
    const float2* tab_w5;  // [tile][view][pair] the fifth ray's weights of both pixels
    const int* tab_la;     // [tile][view][pair] 8 la + n: the first of the pair's five table rays (detector
                           // index la) and how many of them weigh (n <= 5), or kBwdTabOverflow
    const int* tab_vflag;  // [tile][view] nonzero where some pair of the tile overflows in that view
};

// Weight table of the exact adjoint (the TAB mode of the packed kernel): per 16 x 16 tile, view and
// consumer thread (a vertical pixel pair, the PX = 2 layout) the detector index la of the first ray
// that weighs on either pixel and both pixels' weights on rays la .. la + 4 (zero past the pair's
// candidates), or la = kBwdTabOverflow where the pair's weighted rays span more than five detectors
// (rays much denser than a pixel) -- such pairs compute their weights as without a table.  (On the
// 512^2 fan with 720 views and 1024 detectors a pair's weighted rays span 2-5 detectors: five
// covers all but ~0.1 % of the pairs and views, four left ~1.4 % to the slower path, spread over a
// third of the warps.)  The weights are the gather's own: the same re-based ray records and the same
// bwdp_weight arithmetic, so the table adjoint adds the same nonzero products in the same order.
constexpr int kBwdTabRays = 5;
constexpr int kBwdTabOverflow = (int)0x80000000;
constexpr int kBwdTabPairs = kBwdThreads / 2;   // consumer threads of a 16-image CTA

// Pixel pair of consumer thread `tid` in a 16 x 16 tile (PX = 2): rows pi0, pi0 + 1 of column pj.
// Each warp takes an 8 x 8 block, each group of eight lanes a 4 x 4 block (2 x 4 pairs).
__host__ __device__ inline void bwdp_pair_of(int tid, int* pi0, int* pj) {
    const int warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 3, e8 = lane & 7;
    *pi0 = (warp >> 1) * 8 + ((grp >> 1) * 2 + (e8 >> 2)) * 2;
    *pj = (warp & 1) * 8 + (grp & 1) * 4 + (e8 & 3);
}

// Detector window of a tile for one view (bwd_view_window) and the largest detector coordinate of
// its pixels, from the tile's four corners (a linear-fractional map takes its extremes over a
// convex tile at the corners).
__device__ __forceinline__ float bwdp_tile_tmax(const ViewF vf, int ti, int tj, int n) {
    const float x0 = (float)tj, x1 = (float)min(tj + kBwdTile - 1, n - 1);
    const float y0 = (float)ti, y1 = (float)min(ti + kBwdTile - 1, n - 1);
    return fmaxf(fmaxf(bwd_det_coord(vf, x0, y0), bwd_det_coord(vf, x1, y0)),
                 fmaxf(bwd_det_coord(vf, x0, y1), bwd_det_coord(vf, x1, y1)));
}

// Re-based ray record: A = (reference sample relative to the tile origin, step), Bc = (step / h^2,
// C, 0) with C = -A.b - kr, so that the first of a pixel's KW candidate samples is
// ceil(p.b + C) samples past the reference (kr = (|dx| + |dy|) / h^2 + 1e-4 half-widths the window:
// every sample within the pixel's 2 x 2 support lies within kr of the pixel's projection).  A ray
// outside the detector gets a far-away sentinel with step zero (weight zero everywhere).
__device__ __forceinline__ void bwdp_rebase(const RayT ray, bool valid, int ti, int tj, float ih2, float4* A,
                                            float4* Bc) {
    *A = bwd_ray_pos_rec(ray, valid, ti, tj, ih2);
    const float bx = A->z * ih2, by = A->w * ih2;
    const float kr = fmaf(fabsf(A->z) + fabsf(A->w), ih2, 1e-4f);
    *Bc = make_float4(bx, by, -fmaf(A->x, bx, A->y * by) - kr, 0.0f);
}

// Bilinear weight of the pixel at (px, py) (tile-local) on one ray with record A = (reference sample
// relative to the tile origin, step) and Bc = (step / h^2, C): the sum over KW consecutive samples
// from the window start ceil(p.b + C) of tent(dx) * tent(dy), tent(v) = max(0, 1 - |v|) evaluated
// as one saturating add (1 - |v| <= 1, so clamping to [0, 1] only clamps at 0).  `s` is p.b + C.
template <int KW>
__device__ __forceinline__ float bwdp_weight(float px, float py, float s, const float4 A) {
    const float ka = ceilf(s);
    float rx = fmaf(ka, A.z, A.x - px), ry = fmaf(ka, A.w, A.y - py);   // sample ka relative to the pixel
    float w = __saturatef(1.0f - fabsf(rx)) * __saturatef(1.0f - fabsf(ry));
#pragma unroll
    for (int k = 1; k < KW; ++k) {
        rx += A.z;
        ry += A.w;
        w = fmaf(__saturatef(1.0f - fabsf(rx)), __saturatef(1.0f - fabsf(ry)), w);
    }
    return w;
}

// 16-bit row segment of 8 images (one 16-byte load) -> 8 FP32 words (two 16-byte stores).
template <typename T>
__device__ __forceinline__ void bwdp_widen8(const uint4 u, float4* out);

template <>
__device__ __forceinline__ void bwdp_widen8<__half>(const uint4 u, float4* out) {
    __half2 h[4];
    memcpy(h, &u, 16);
    const float2 a = __half22float2(h[0]), b = __half22float2(h[1]), c = __half22float2(h[2]),
                 d = __half22float2(h[3]);
    out[0] = make_float4(a.x, a.y, b.x, b.y);
    out[1] = make_float4(c.x, c.y, d.x, d.y);
}

template <>
__device__ __forceinline__ void bwdp_widen8<__nv_bfloat16>(const uint4 u, float4* out) {
    out[0] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                         __uint_as_float(u.y & 0xffff0000u));
    out[1] = make_float4(__uint_as_float(u.z << 16), __uint_as_float(u.z & 0xffff0000u), __uint_as_float(u.w << 16),
                         __uint_as_float(u.w & 0xffff0000u));
}

// TAB (exact adjoint, PX = 2 only): a pair's weights come from the geometry's weight table instead of
// being evaluated from re-based ray records; ray rows are copied and re-based only for chunks with a
// view in which some pair of the tile overflows the table (the table's per-view flags).  The producer
// prefetches the table's rows for the chunk that will next reuse its ring slot into L2.
template <typename T, int BG, int KW, bool TAB = false>
__global__ void __launch_bounds__(BwdPShape<BG>::kThreads, BwdPShape<BG>::kCtasPerSm)
    backward_packed_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap rmap,
                           const BwdPArgs a) {
    static_assert(!TAB || (KW > 0 && BwdPShape<BG>::PX == 2), "the weight table serves the exact adjoint's pairs");
    constexpr bool kRays = KW > 0;   // ray rows copied and re-based per chunk
    using L = BwdPLayout<T, BG>;
    constexpr int NQ = BG / 4;
    constexpr int PITCH = L::kPitch;
    constexpr int PX = BwdPShape<BG>::PX;
    constexpr int NC = BwdPShape<BG>::kConsumers;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* tma_bar = reinterpret_cast<uint64_t*>(smem);        // [stages]: a slot's copies landed
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + 64);     // [stages]: consumers released a slot
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 128);
    int* dlo_c = reinterpret_cast<int*>(smem + 192);              // [stages][views]
    float* r_c = reinterpret_cast<float*>(smem + 256);            // [stages][views]
    ViewF* view_c = reinterpret_cast<ViewF*>(smem + 512);         // [stages][views]
    int* rays_c = reinterpret_cast<int*>(smem + 320);             // [stages]: the chunk's ray rows were copied
    static_assert(kBwdPMaxStages * kBwdPViews * 4 <= 64 && 512 + kBwdPMaxStages * kBwdPViews * 32 <= kBwdPHeader,
                  "ring header overflows its slots");
    const int S = a.stages;
    const BwdPSmem m = bwdp_smem<T, BG>(a.wd, S, kRays);
    unsigned char* ring = smem + kBwdPHeader;
    unsigned char* yf = ring + (size_t)S * m.stage;   // [2][views] converted windows (16-bit storage)

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int ti = (tile / a.tiles_x) * kBwdTile, tj = (tile - (tile / a.tiles_x) * a.tiles_x) * kBwdTile;
    const int nchunks = (a.V + kBwdPViews - 1) / kBwdPViews;

    if (tid < S) {
        mbar_init(&tma_bar[tid], 1);
        mbar_init(&empty[tid], NC);
    }
    if (tid == 0) *abort_flag = 0;
    fence_mbar_init();
    __syncthreads();

    if (tid >= NC) {
        // ------------------------------------------------------------------ producer warp
        const int lane = tid & 31;
        int c = 0;
        for (; c < nchunks; ++c) {
            const int st = c % S;
            bool ok = true;
            if (c >= S && lane == 0) ok = mbar_wait_bounded(&empty[st], (uint32_t)((c / S - 1) & 1), a.spin_limit);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            const int v0 = c * kBwdPViews;
            const int nv = min(kBwdPViews, a.V - v0);
            if (lane < nv) {
                const ViewF vf = a.views[v0 + lane];
                int dlo;
                float r;
                bwd_view_window(vf, ti, tj, a.n, &dlo, &r);
                // every pixel's candidates [ceil(t - r), floor(t + r)] within the detector must lie in
                // the copied window; the consumers clamp to it, so a miss is recorded, not overrun
                const float thi = floorf(bwdp_tile_tmax(vf, ti, tj, a.n) + r);
                if (fminf(thi, (float)(a.D - 1)) > (float)(dlo + a.wd - 1)) record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
                dlo_c[st * kBwdPViews + lane] = dlo;
                r_c[st * kBwdPViews + lane] = r;
                view_c[st * kBwdPViews + lane] = vf;
            }
            // ray rows: always for the on-the-fly weights; with a table only where some pair overflows
            bool rays = kRays;
            if constexpr (TAB) {
                const int fl = lane < nv ? __ldg(a.tab_vflag + (size_t)tile * a.V + v0 + lane) : 0;
                rays = __any_sync(0xffffffffu, fl != 0);
            }
            __syncwarp();
            if (lane == 0) {
                unsigned char* slot = ring + (size_t)st * m.stage;
                rays_c[st] = rays ? 1 : 0;
                fence_proxy_async_shared();
                mbar_arrive_expect_tx(&tma_bar[st],
                                      (uint32_t)(nv * a.wd * (L::kRowElems * (int)sizeof(T) + (rays ? 32 : 0))));
                for (int vl = 0; vl < nv; ++vl) {
                    const int dlo = dlo_c[st * kBwdPViews + vl];
                    tma_load_4d(slot + (size_t)vl * m.yst_view, &map, &tma_bar[st], 0, dlo, v0 + vl, blockIdx.y);
                    if (rays)   // the interpolating backprojector needs no rays
                        tma_load_2d(slot + (size_t)kBwdPViews * m.yst_view + (size_t)vl * m.rst_view, &rmap,
                                    &tma_bar[st], 0, (v0 + vl) * a.D + dlo);
                }
                if constexpr (TAB) {
                    // the table rows of the chunk that will next use this slot, into L2 (a hint: no
                    // completion to wait for); 16-byte aligned multiples of 16 bytes by construction
                    const int cn = c + S;
                    if (cn < nchunks) {
                        const int vn = cn * kBwdPViews, nvn = min(kBwdPViews, a.V - vn);
                        const size_t rec = ((size_t)tile * a.V + vn) * kBwdTabPairs;
                        bulk_prefetch_l2(a.tab_w + 2 * rec, (uint32_t)(nvn * kBwdTabPairs * 32));
                        bulk_prefetch_l2(a.tab_w5 + rec, (uint32_t)(nvn * kBwdTabPairs * 8));
                        bulk_prefetch_l2(a.tab_la + rec, (uint32_t)(nvn * kBwdTabPairs * 4));
                    }
                }
            }
            __syncwarp();
        }
        if (c < nchunks && lane == 0) {
            // The consumers stopped releasing slots: record it, let the copies still in flight land
            // (bounded), then complete chunk c's phase without data so any consumer still waiting
            // sees the abort.
            record_device_error(a.err, RADON_ERR_TIMEOUT);
            *abort_flag = 1;
            for (int cc = max(0, c - S + 1); cc < c; ++cc)
                mbar_wait_bounded(&tma_bar[cc % S], (uint32_t)((cc / S) & 1), a.spin_limit);
            mbar_arrive(&tma_bar[c % S]);
        }
        return;
    }

    // ---------------------------------------------------------------------- consumer warps
    // each warp takes an (4 PX) x 8 block of the tile, lanes on a 4 x 8 grid of pixels (PX = 1) or
    // vertical pixel pairs (PX = 2): a block's detector footprints overlap more than those of a strip,
    // so the gather's shared loads touch fewer distinct addresses.  A 16-byte shared load is served
    // eight lanes at a time, so each group of eight lanes covers a compact block -- 4 x 2 pixels, or
    // 2 x 4 pairs (4 x 4 pixels) -- whose detector span stays within the eight bank groups
    const int warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 3, e8 = lane & 7;
    int pi0 = (warp >> 1) * 4 + (e8 >> 1), pj = (warp & 1) * 8 + grp * 2 + (e8 & 1);
    if constexpr (PX == 2) bwdp_pair_of(tid, &pi0, &pj);
    const float px = (float)pj, py0 = (float)pi0;
    const float gx = (float)(tj + pj), gy0 = (float)(ti + pi0);
    float acc[PX][BG];
#pragma unroll
    for (int x = 0; x < PX; ++x)
#pragma unroll
        for (int b = 0; b < BG; ++b) acc[x][b] = 0.0f;
    constexpr int OCT = BG / 8;                 // 16-byte segments of a 16-bit window row
    constexpr int LOG_OCT = OCT == 1 ? 0 : OCT == 2 ? 1 : 2;
    const uint32_t ring_a = smem_u32(ring), yf_a = smem_u32(yf);
    const uint32_t win_a = smem_u32(view_c);
    const uint32_t yview = L::kConv ? (uint32_t)m.yf_view : (uint32_t)m.yst_view;
    const uint32_t ystv = (uint32_t)m.yst_view, rstv = (uint32_t)m.rst_view;
    // TAB: this thread's table record of the next view, loaded one view ahead of its use
    [[maybe_unused]] float4 tw0 = make_float4(0.f, 0.f, 0.f, 0.f), tw1 = tw0;
    [[maybe_unused]] float2 tw5 = make_float2(0.f, 0.f);
    [[maybe_unused]] int tla = 0;
    [[maybe_unused]] const size_t trec0 = (size_t)tile * a.V * kBwdTabPairs + (size_t)tid;
    if constexpr (TAB) {
        tw0 = __ldg(a.tab_w + 2 * trec0);
        tw1 = __ldg(a.tab_w + 2 * trec0 + 1);
        tw5 = __ldg(a.tab_w5 + trec0);
        tla = __ldg(a.tab_la + trec0);
    }
    for (int c = 0; c < nchunks; ++c) {
        const int st = c % S;
        const int v0 = c * kBwdPViews;
        const int nv = min(kBwdPViews, a.V - v0);
        bool bad = !mbar_wait_bounded(&tma_bar[st], (uint32_t)((c / S) & 1), a.spin_limit);
        bad = bad || *abort_flag != 0;
        const uint32_t slot_a = ring_a + (uint32_t)st * (uint32_t)m.stage;
        const uint32_t rst_a = slot_a + kBwdPViews * ystv;
        const uint32_t ybuf_a = L::kConv ? yf_a + (uint32_t)(c & 1) * (uint32_t)m.yf_buf : slot_a;
        if (!bad) {
            // (the table gather converts the 16-bit rows it reads itself: the widened rows serve only
            // the on-the-fly weights, needed where the chunk's rays were copied)
            if (L::kConv && (!TAB || rays_c[st])) {
                // 16-bit window rows -> FP32 rows of pitch PITCH (8 images per 16-byte load); the
                // view of item e is found by comparison (no division)
                const int W = a.wd * OCT;
                for (int e = tid; e < nv * W; e += NC) {
                    int vl = 0;
#pragma unroll
                    for (int m = 1; m < kBwdPViews; ++m) vl += e >= m * W;
                    const int rest = e - vl * W;
                    const int dl = rest >> LOG_OCT, o = rest & (OCT - 1);
                    const uint4 u = lds4u(slot_a + (uint32_t)vl * ystv + (uint32_t)(dl * BG * 2 + o * 16));
                    float4 f[2];
                    bwdp_widen8<T>(u, f);
                    const uint32_t dst = ybuf_a + (uint32_t)vl * yview + (uint32_t)(dl * PITCH + o * 32);
                    sts4(dst, f[0]);
                    sts4(dst + 16, f[1]);
                }
            }
            if (kRays && rays_c[st]) {
                // re-base the landed rays on this tile, in place: one ray per thread
                const int W = a.wd;
                for (int e = tid; e < nv * W; e += NC) {
                    int vl = 0;
#pragma unroll
                    for (int m = 1; m < kBwdPViews; ++m) vl += e >= m * W;
                    const int dl = e - vl * W;
                    const int d = dlo_c[st * kBwdPViews + vl] + dl;
                    const uint32_t rec = rst_a + (uint32_t)vl * rstv + (uint32_t)dl * 32u;
                    const float4 lo = lds4(rec), hi = lds4(rec + 16);
                    RayT ray;
                    ray.J0 = __float_as_int(lo.x);
                    ray.I0 = __float_as_int(lo.y);
                    ray.fx0 = lo.z;
                    ray.fy0 = lo.w;
                    ray.dxh = hi.x;
                    ray.dyh = hi.y;
                    ray.dxl = hi.z;
                    ray.dyl = hi.w;
                    float4 A, Bc;
                    bwdp_rebase(ray, d >= 0 && d < a.D, ti, tj, a.ih2, &A, &Bc);
                    sts4(rec, A);
                    sts4(rec + 16, Bc);
                }
            }
        }
        // all consumers: windows and records written (the converted buffer alternates, so the
        // previous chunk's readers have all passed this barrier before it is overwritten) -- and
        // one shared abort decision
        if (named_barrier_or(1, NC, bad)) {
            if (tid == 0) record_device_error(a.err, RADON_ERR_TIMEOUT);
            return;
        }
        for (int vl = 0; vl < nv; ++vl) {
            const uint32_t va = win_a + (uint32_t)(st * kBwdPViews + vl) * 32u;
            const float4 v01 = lds4(va), v23 = lds4(va + 16);   // ax, ay, a0, bx | by, b0, -, -
            const int dlo = dlo_c[st * kBwdPViews + vl];
            const uint32_t yv = ybuf_a + (uint32_t)vl * yview;
            // detector coordinate of the first pixel; the second (one row down) adds (ay, by)
            const float num0 = fmaf(v01.x, gx, fmaf(v01.y, gy0, v01.z));
            const float den0 = fmaf(v01.w, gx, fmaf(v23.x, gy0, v23.y));
            if constexpr (KW == 0) {
                // interpolating backprojector: the sinogram linearly interpolated at the pixel's detector
                // coordinate t (IEEE division: the weights need t to ~1e-5 bins), weighted by the ray
                // density |grad t|; both taps lie in the copied window by construction of its bounds
                const int lo = max(dlo, 0) - dlo, hi = min(a.D - 1, dlo + a.wd - 1) - dlo;
#pragma unroll
                for (int x = 0; x < PX; ++x) {
                    const float gy = gy0 + (float)x;
                    const float den = fmaf(v01.w, gx, fmaf(v23.x, gy, v23.y));
                    const float t = fmaf(v01.x, gx, fmaf(v01.y, gy, v01.z)) / den;
                    const float ga = fmaf(-t, v01.w, v01.x), gb = fmaf(-t, v23.x, v01.y);
                    const float w = sqrtf(fmaf(ga, ga, gb * gb)) / fabsf(den);
                    const float fl = floorf(t);
                    const int k = (int)fl - dlo;
                    const float f = t - fl;
                    const float w0 = w * (1.0f - f), w1 = w * f;
                    const bool in0 = k >= lo && k <= hi, in1 = k + 1 >= lo && k + 1 <= hi;
                    const uint32_t y0 = yv + (uint32_t)k * PITCH;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (in0) {
                            const float4 y4 = lds4(y0 + 16 * q);
                            acc[x][4 * q + 0] = fmaf(w0, y4.x, acc[x][4 * q + 0]);
                            acc[x][4 * q + 1] = fmaf(w0, y4.y, acc[x][4 * q + 1]);
                            acc[x][4 * q + 2] = fmaf(w0, y4.z, acc[x][4 * q + 2]);
                            acc[x][4 * q + 3] = fmaf(w0, y4.w, acc[x][4 * q + 3]);
                        }
                        if (in1) {
                            const float4 y4 = lds4(y0 + PITCH + 16 * q);
                            acc[x][4 * q + 0] = fmaf(w1, y4.x, acc[x][4 * q + 0]);
                            acc[x][4 * q + 1] = fmaf(w1, y4.y, acc[x][4 * q + 1]);
                            acc[x][4 * q + 2] = fmaf(w1, y4.z, acc[x][4 * q + 2]);
                            acc[x][4 * q + 3] = fmaf(w1, y4.w, acc[x][4 * q + 3]);
                        }
                    }
                }
            } else {
                bool tabbed = false;
                if constexpr (TAB) {
                    // the pair's table rays from la: rows clamped into the window (a clamped row has
                    // weight zero); the same nonzero products, in the same order, as the gather.  The
                    // warp runs to the largest count of weighted rays among its pairs (the rest of a
                    // pair's five carry zero weight)
                    const float4 w0 = tw0, w1 = tw1;
                    const float2 w5 = tw5;
                    const int pk = tla;
                    const bool over_t = pk == kBwdTabOverflow;
                    const int la_t = pk >> 3;
                    const int nc = __reduce_max_sync(0xffffffffu, over_t ? 0 : (pk & 7));
                    const int vnext = v0 + vl + 1;
                    if (vnext < a.V) {
                        const size_t nr = trec0 + (size_t)vnext * kBwdTabPairs;
                        tw0 = __ldg(a.tab_w + 2 * nr);
                        tw1 = __ldg(a.tab_w + 2 * nr + 1);
                        tw5 = __ldg(a.tab_w5 + nr);
                        tla = __ldg(a.tab_la + nr);
                    }
                    if (!over_t) {
                        tabbed = true;
                        const int rel0 = la_t - dlo;
                        const float wa[kBwdTabRays] = {w0.x, w0.y, w0.z, w0.w, w5.x};
                        const float wb[kBwdTabRays] = {w1.x, w1.y, w1.z, w1.w, w5.y};
#pragma unroll
                        for (int cr = 0; cr < kBwdTabRays; ++cr) {
                            if (cr >= nc) break;
                            const int rel = min(max(rel0 + cr, 0), a.wd - 1);
                            // 16-bit storage: the landed row itself, converted in registers (half the
                            // shared loads of the widened row, and no widening pass); FP32: the row
                            const uint32_t ya = yv + (uint32_t)rel * PITCH;
                            const uint32_t yr = slot_a + (uint32_t)vl * ystv + (uint32_t)rel * (uint32_t)(BG * 2);
                            float4 yw[NQ];
                            if constexpr (L::kConv) {
#pragma unroll
                                for (int o = 0; o < NQ / 2; ++o) {
                                    float4 f[2];
                                    bwdp_widen8<T>(lds4u(yr + 16 * o), f);
                                    yw[2 * o] = f[0];
                                    yw[2 * o + 1] = f[1];
                                }
                            }
                            // paired FMAs (two images per fma.rn.f32x2, each lane an IEEE fma: the same
                            // bits as scalar FMAs, half the FMA instructions)
                            const f32x2 wwa = f2_pack(wa[cr], wa[cr]), wwb = f2_pack(wb[cr], wb[cr]);
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                float4 y4;
                                if constexpr (L::kConv) y4 = yw[q];
                                else y4 = lds4(ya + 16 * q);
                                const f32x2 y01 = f2_pack(y4.x, y4.y), y23 = f2_pack(y4.z, y4.w);
                                f32x2 a0 = f2_pack(acc[0][4 * q + 0], acc[0][4 * q + 1]);
                                f32x2 a1 = f2_pack(acc[0][4 * q + 2], acc[0][4 * q + 3]);
                                f32x2 b0 = f2_pack(acc[PX - 1][4 * q + 0], acc[PX - 1][4 * q + 1]);
                                f32x2 b1 = f2_pack(acc[PX - 1][4 * q + 2], acc[PX - 1][4 * q + 3]);
                                a0 = f2_fma(wwa, y01, a0);
                                a1 = f2_fma(wwa, y23, a1);
                                b0 = f2_fma(wwb, y01, b0);
                                b1 = f2_fma(wwb, y23, b1);
                                f2_unpack(a0, &acc[0][4 * q + 0], &acc[0][4 * q + 1]);
                                f2_unpack(a1, &acc[0][4 * q + 2], &acc[0][4 * q + 3]);
                                f2_unpack(b0, &acc[PX - 1][4 * q + 0], &acc[PX - 1][4 * q + 1]);
                                f2_unpack(b1, &acc[PX - 1][4 * q + 2], &acc[PX - 1][4 * q + 3]);
                            }
                        }
                    }
                }
                if (!tabbed) {
                    const float r = r_c[st * kBwdPViews + vl];
                    // the union of the pixels' candidate ranges [t - r, t + r] (approximate divide: the
                    // windows carry margins far above its error); a candidate outside a pixel's own range
                    // has zero weight there.  Candidates outside the detector are sentinel rays over
                    // zero-filled rows, so only the copied window bounds the loop (the producer checked
                    // that it holds them all); the bounds are clamped in FP32, so a non-finite coordinate
                    // still gives a loop inside the window
                    float tlo = __fdividef(num0, den0), thi = tlo;
                    if constexpr (PX == 2) {
                        const float t1 = __fdividef(num0 + v01.y, den0 + v23.x);
                        tlo = fminf(tlo, t1);
                        thi = fmaxf(thi, t1);
                    }
                    const float fd = (float)dlo;
                    const int la = __float2int_ru(fmaxf((tlo - r) - fd, 0.0f));
                    const int lb = __float2int_rd(fminf((thi + r) - fd, (float)(a.wd - 1)));
                    uint32_t ra = rst_a + (uint32_t)vl * rstv + (uint32_t)la * 32u;
                    uint32_t ya = yv + (uint32_t)la * PITCH;
                    for (int dl = la; dl <= lb; ++dl, ra += 32u, ya += PITCH) {
                        const float4 A = lds4(ra), Bc = lds4(ra + 16);
                        const float s0 = fmaf(px, Bc.x, fmaf(py0, Bc.y, Bc.z));
                        float w[PX];
                        w[0] = bwdp_weight<KW>(px, py0, s0, A);
                        if constexpr (PX == 2) w[1] = bwdp_weight<KW>(px, py0 + 1.0f, s0 + Bc.y, A);
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            const float4 y4 = lds4(ya + 16 * q);
                            if constexpr (PX == 2) {
                                // pixel pairs: paired FMAs (the same bits as scalar ones; measured 2-3 %
                                // faster here, while the 32-image groups' single pixels ran slower paired)
                                const f32x2 y01 = f2_pack(y4.x, y4.y), y23 = f2_pack(y4.z, y4.w);
#pragma unroll
                                for (int x = 0; x < PX; ++x) {
                                    const f32x2 ww = f2_pack(w[x], w[x]);
                                    f32x2 a0 = f2_pack(acc[x][4 * q + 0], acc[x][4 * q + 1]);
                                    f32x2 a1 = f2_pack(acc[x][4 * q + 2], acc[x][4 * q + 3]);
                                    a0 = f2_fma(ww, y01, a0);
                                    a1 = f2_fma(ww, y23, a1);
                                    f2_unpack(a0, &acc[x][4 * q + 0], &acc[x][4 * q + 1]);
                                    f2_unpack(a1, &acc[x][4 * q + 2], &acc[x][4 * q + 3]);
                                }
                            } else {
#pragma unroll
                                for (int x = 0; x < PX; ++x) {
                                    acc[x][4 * q + 0] = fmaf(w[x], y4.x, acc[x][4 * q + 0]);
                                    acc[x][4 * q + 1] = fmaf(w[x], y4.y, acc[x][4 * q + 1]);
                                    acc[x][4 * q + 2] = fmaf(w[x], y4.z, acc[x][4 * q + 2]);
                                    acc[x][4 * q + 3] = fmaf(w[x], y4.w, acc[x][4 * q + 3]);
                                }
                            }
                        }
                    }
                }
            }
        }
        mbar_arrive(&empty[st]);
    }
    const long long npix = (long long)a.n * a.n;
    const int b0 = blockIdx.y * BG;
#pragma unroll
    for (int x = 0; x < PX; ++x) {
        if ((ti + pi0 + x) >= a.n || (tj + pj) >= a.n) continue;
        const long long p = (long long)(ti + pi0 + x) * a.n + (tj + pj);
#pragma unroll
        for (int b = 0; b < BG; ++b)
            if (b0 + b < a.B)
                epilogue_store_rt(a.ep, a.out_dtype, a.img, a.h * acc[x][b], (long long)(b0 + b) * npix + p);
    }
}

// Builds the weight table of the exact adjoint: one CTA per (tile, block of views), one thread per
// consumer pixel pair (bwdp_pair_of).  For each view the thread takes the pair's candidate rays as the
// gather does (the tile's window, the union of the pixels' ranges [t - r, t + r] clamped to it),
// re-bases each on the tile and evaluates both pixels' weights with bwdp_weight; it stores the first
// ray that weighs on either pixel (la), the count of weighted rays from it and the weights on rays
// la .. la + 4 (record 8 la + count), or kBwdTabOverflow where
// the weighted rays span more than five (counted in *overflow, and flagged for the tile and view in
// tab_vflag, which must start at zero).
template <int KW>
__global__ void __launch_bounds__(kBwdTabPairs) bwdp_table_kernel(const RayT* __restrict__ rays,
                                                                 const ViewF* __restrict__ views, int n, int V, int D,
                                                                 float ih2, int wd, int tiles_x, int views_per_block,
                                                                 float4* __restrict__ tab_w, float2* __restrict__ tab_w5,
                                                                 int* __restrict__ tab_la, int* __restrict__ tab_vflag,
                                                                 unsigned long long* overflow) {
    const int tile = blockIdx.x, tid = threadIdx.x;
    const int ti = (tile / tiles_x) * kBwdTile, tj = (tile - (tile / tiles_x) * tiles_x) * kBwdTile;
    int pi0, pj;
    bwdp_pair_of(tid, &pi0, &pj);
    const float px = (float)pj, py0 = (float)pi0;
    const float gx = (float)(tj + pj), gy0 = (float)(ti + pi0);
    const int vb = blockIdx.y * views_per_block, ve = min(vb + views_per_block, V);
    for (int v = vb; v < ve; ++v) {
        const ViewF vf = views[v];
        int dlo;
        float r;
        bwd_view_window(vf, ti, tj, n, &dlo, &r);
        const float num0 = fmaf(vf.ax, gx, fmaf(vf.ay, gy0, vf.a0));
        const float den0 = fmaf(vf.bx, gx, fmaf(vf.by, gy0, vf.b0));
        float tlo = __fdividef(num0, den0), thi = tlo;
        const float t1 = __fdividef(num0 + vf.ay, den0 + vf.by);
        tlo = fminf(tlo, t1);
        thi = fmaxf(thi, t1);
        const float fd = (float)dlo;
        const int la = __float2int_ru(fmaxf((tlo - r) - fd, 0.0f));
        const int lb = __float2int_rd(fminf((thi + r) - fd, (float)(wd - 1)));
        auto weights = [&](int dl, float* w0, float* w1) {
            const int d = dlo + dl;
            const bool valid = d >= 0 && d < D;
            RayT ray{0, 0, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (valid) ray = rays[(long long)v * D + d];
            float4 A, Bc;
            bwdp_rebase(ray, valid, ti, tj, ih2, &A, &Bc);
            const float s0 = fmaf(px, Bc.x, fmaf(py0, Bc.y, Bc.z));
            *w0 = bwdp_weight<KW>(px, py0, s0, A);
            *w1 = bwdp_weight<KW>(px, py0 + 1.0f, s0 + Bc.y, A);
        };
        int f = -1, l = -1;
        for (int dl = la; dl <= lb; ++dl) {
            float w0, w1;
            weights(dl, &w0, &w1);
            if (w0 != 0.0f || w1 != 0.0f) {
                if (f < 0) f = dl;
                l = dl;
            }
        }
        const bool over = f >= 0 && l - f >= kBwdTabRays;
        if (over) {
            atomicAdd(overflow, 1ull);
            atomicOr(tab_vflag + (size_t)tile * V + v, 1);
        }
        const int first = f >= 0 ? f : la;
        float wa[kBwdTabRays], wb[kBwdTabRays];
#pragma unroll
        for (int cr = 0; cr < kBwdTabRays; ++cr) {
            wa[cr] = 0.0f;
            wb[cr] = 0.0f;
            const int dl = first + cr;
            if (!over && dl >= la && dl <= lb) weights(dl, &wa[cr], &wb[cr]);
        }
        const size_t rec = ((size_t)tile * V + v) * kBwdTabPairs + tid;
        tab_w[2 * rec] = make_float4(wa[0], wa[1], wa[2], wa[3]);
        tab_w[2 * rec + 1] = make_float4(wb[0], wb[1], wb[2], wb[3]);
        tab_w5[rec] = make_float2(wa[4], wb[4]);
        tab_la[rec] = over ? kBwdTabOverflow : (dlo + first) * 8 + (f >= 0 ? l - f + 1 : 0);
    }
}

// Ring depth of a packed-adjoint CTA: the deepest ring (up to kBwdPMaxStages) that keeps the launch
// bounds' CTAs resident per SM (228 KB of shared memory, 1 KB reserved per CTA), else two stages;
// returns the dynamic shared memory.
template <typename T, int BG>
inline size_t bwdp_plan(int wd, bool rays, int* stages) {
    const size_t budget = (size_t)228 * 1024 / BwdPShape<BG>::kCtasPerSm - 1024;
    int S = kBwdPMaxStages;
    while (S > 2 && bwdp_smem<T, BG>(wd, S, rays).total > budget) --S;
    *stages = S;
    return bwdp_smem<T, BG>(wd, S, rays).total;
}

template <typename T, int BG, int KW, bool TAB = false>
cudaError_t bwdp_launch(const CUtensorMap& map, const CUtensorMap& rmap, const BwdPArgs& a, dim3 grid, size_t smem,
                        cudaStream_t s) {
    auto kern = backward_packed_kernel<T, BG, KW, TAB>;
    static size_t attr_bytes = 0;
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    kern<<<grid, BwdPShape<BG>::kThreads, smem, s>>>(map, rmap, a);
    return cudaGetLastError();
}

// Host launcher for storage type T and BG images per CTA (backward_packed_{f32,f16,bf16}.cu
// instantiate it): `packed` holds pack_sino's rows for this batch; kw = 0 runs the interpolating
// backprojector, 3 or 6 the exact adjoint with that many samples per candidate window.
template <typename T, int BG>
radon_status launch_backward_packed_t(const radon_geometry* g, const void* packed, void* img, radon_dtype dt,
                                      int batch, int kw, const Epilogue& ep, cudaStream_t s, std::string* why,
                                      const CUtensorMap& rmap, uint32_t spin_limit, int* err) {
    using L = BwdPLayout<T, BG>;
    const int wd = g->bwd_window + 2;
    if (wd > 256) {
        *why = "detector window wider than a TMA box";
        return RADON_ERR_UNSUPPORTED;
    }
    // the geometry's weight table serves the exact adjoint's pixel pairs (16-bit or smaller groups)
    const bool tab = kw > 0 && BwdPShape<BG>::PX == 2 && g->d_tab_w != nullptr && g->tab_kw == kw && g->tab_wd == wd;
    int stages = 2;
    // the table kernel stages ray rows too (for the pairs its table marks as overflowing)
    const size_t smem = bwdp_plan<T, BG>(wd, kw > 0, &stages);
    if (smem > 227 * 1024) {
        *why = "shared memory budget exceeded";
        return RADON_ERR_UNSUPPORTED;
    }
    const int groups = (batch + BG - 1) / BG;
    const uint64_t row = (uint64_t)L::kRowElems * sizeof(T);
    const uint64_t dims[4] = {(uint64_t)L::kRowElems, (uint64_t)g->D, (uint64_t)g->V, (uint64_t)groups};
    const uint64_t strides[3] = {row, row * (uint64_t)g->D, row * (uint64_t)g->D * (uint64_t)g->V};
    const uint32_t box[4] = {(uint32_t)L::kRowElems, (uint32_t)wd, 1, 1};
    CUtensorMap map;
    const int rc = encode_tiled(&map, tma_dtype(dt), 4, const_cast<void*>(packed), dims, strides, box,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
    if (rc != 0) {
        *why = "cuTensorMapEncodeTiled rejected the packed-sinogram descriptor (CUresult " + std::to_string(rc) + ")";
        return RADON_ERR_UNSUPPORTED;
    }
    BwdPArgs a;
    a.views = g->d_view;
    a.img = img;
    a.n = g->n;
    a.V = g->V;
    a.D = g->D;
    a.B = batch;
    a.h = kw == 0 ? 1.0f : (float)g->h;   // the interpolating backprojector's sum carries no step factor
    a.ih2 = (float)(1.0 / (g->h * g->h));
    a.wd = wd;
    a.stages = stages;
    a.tiles_x = (g->n + kBwdTile - 1) / kBwdTile;
    a.out_dtype = dt;
    a.err = err;
    a.spin_limit = spin_limit;
    a.ep = ep;
    a.tab_w = static_cast<const float4*>(g->d_tab_w);
    a.tab_w5 = static_cast<const float2*>(g->d_tab_w5);
    a.tab_vflag = g->d_tab_vflag;
    a.tab_la = g->d_tab_la;
    const dim3 grid((unsigned)(a.tiles_x * a.tiles_x), (unsigned)groups);
    cudaError_t e;
    if constexpr (BwdPShape<BG>::PX == 2) {
        if (tab) {
            e = kw == 3 ? bwdp_launch<T, BG, 3, true>(map, rmap, a, grid, smem, s)
                        : bwdp_launch<T, BG, 6, true>(map, rmap, a, grid, smem, s);
        } else {
            e = kw == 0   ? bwdp_launch<T, BG, 0>(map, rmap, a, grid, smem, s)
                : kw == 3 ? bwdp_launch<T, BG, 3>(map, rmap, a, grid, smem, s)
                          : bwdp_launch<T, BG, 6>(map, rmap, a, grid, smem, s);
        }
    } else {
        e = kw == 0   ? bwdp_launch<T, BG, 0>(map, rmap, a, grid, smem, s)
            : kw == 3 ? bwdp_launch<T, BG, 3>(map, rmap, a, grid, smem, s)
                      : bwdp_launch<T, BG, 6>(map, rmap, a, grid, smem, s);
    }
    if (e != cudaSuccess) {
        *why = std::string("packed adjoint launch: ") + cudaGetErrorString(e);
        return RADON_ERR_CUDA;
    }
    return RADON_OK;
}

}  // namespace radon
