// Staged forward projection of single images (the uneven-batch plan), Section 3.1's ray-driven
// bilinear sampling with the image streamed through shared memory.
//
// Every image is packed once into quad texels (the 2 x 2 neighbourhood of a pixel, see Quad<T>), in
// its own frame and transposed, with two texels of zero border on every side and an even row pitch,
// so that any run of an even number of texels starting at an even column is a 16-byte aligned,
// 16-byte sized block of global memory.
//
// A work item is a group of G consecutive views of one orientation class x Dt detectors (G * Dt * L
// = 256 consumer threads, L lanes per ray).  The CTA streams the compute frame of its class -- rows
// of the image for rays running mostly along y, rows of the transposed image otherwise, so every ray
// advances monotonically through them -- in slabs of R texel rows:
//   * the producer warp bounds slab s's band (the columns crossed by the lines of the item's extreme
//     rays, which enclose every ray of the item) and copies its rows with one bulk copy (TMA,
//     cp.async.bulk) per row into a ring buffer, announcing the bytes on the buffer's full mbarrier;
//     a header beside the buffer names the work item, the slab and the band origin;
//   * the 8 consumer warps wait for a full buffer, march their rays through the slab -- one 8-byte
//     (16-bit storage) or 16-byte (FP32) shared load per sample fetches all four texels -- and
//     release the buffer on its empty mbarrier.
// The producer streams work items back to back (a persistent CTA takes the next item from a device
// counter), so the ring does not drain between items.  Slabs whose band misses the support are never
// copied.  All waits are bounded; on expiry the kernel records RADON_ERR_TIMEOUT and unwinds.
#pragma once

namespace radon {

constexpr int kSfConsumerWarps = 8;
constexpr int kSfConsumers = kSfConsumerWarps * 32;
constexpr int kSfThreads = kSfConsumers + 32;
constexpr int kSfMaxStages = 4;
constexpr int kSfHeaderInts = 8;

// Header flags of a ring buffer.
constexpr int kSfFirst = 1;    // the item's first slab (consumers load their rays)
constexpr int kSfLast = 2;     // the item's last slab (consumers store their sums)
constexpr int kSfNoData = 4;   // nothing was copied (an item whose rays all miss the image)

// Quad texel layout: per frame (n + 3) rows x P columns; texel (r, c), r, c in [-2, n], at
// (r + 2) * P + (c + 2).  P is even and at least n + 4.
__host__ __device__ inline int sq_pitch(int n) { return (n + 5) & ~1; }
__host__ __device__ inline long long sq_frame(int n) { return (long long)(n + 3) * sq_pitch(n); }

// Bulk copy of `bytes` (a multiple of 16) from global `src` to shared `dst` (both 16-byte aligned),
// completing on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint2 lds2u(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

// One quad texel from shared memory as four FP32 values (compute-frame order (r, c), (r, c + 1),
// (r + 1, c), (r + 1, c + 1)).
template <typename T>
__device__ __forceinline__ void sq_load(uint32_t a, float* t);
template <>
__device__ __forceinline__ void sq_load<float>(uint32_t a, float* t) {
    const uint4 q = lds4u(a);
    t[0] = __uint_as_float(q.x);
    t[1] = __uint_as_float(q.y);
    t[2] = __uint_as_float(q.z);
    t[3] = __uint_as_float(q.w);
}
template <>
__device__ __forceinline__ void sq_load<__half>(uint32_t a, float* t) {
    const uint2 q = lds2u(a);
    Quad<__half>::unpack(q, t);
}
template <>
__device__ __forceinline__ void sq_load<__nv_bfloat16>(uint32_t a, float* t) {
    const uint2 q = lds2u(a);
    Quad<__nv_bfloat16>::unpack(q, t);
}

// Quad texel e of a unit's packed image (both frames, the layout above).
template <typename T>
__device__ __forceinline__ typename Quad<T>::type sq_texel(const T* x, int n, long long e) {
    const long long P = sq_pitch(n), F = sq_frame(n);
    const int frame = e >= F ? 1 : 0;
    if (frame) e -= F;
    const int r = (int)(e / P) - 2, c = (int)(e - (e / P) * P) - 2;
    return frame == 0 ? Quad<T>::make(pix(x, n, r, c), pix(x, n, r, c + 1), pix(x, n, r + 1, c), pix(x, n, r + 1, c + 1))
                      : Quad<T>::make(pix(x, n, c, r), pix(x, n, c + 1, r), pix(x, n, c, r + 1), pix(x, n, c + 1, r + 1));
}

struct SfArgs {
    const Unit* units;    // unit table
    const Work* work;     // work list
    int n_work;
    unsigned* counter;    // work counter (zero at launch)
    const void* quads;    // packed quad texels of every unit
    int wbox;             // band columns (even for 16-bit storage)
    int pitch;            // shared row pitch in texels (sf_pitch)
    int rmax;             // rows per slab of the widest unit (buffer rows)
    int stages;           // ring buffers (2..4)
    int* err;
    uint32_t spin_limit;
    Epilogue ep;
};

// Work item `tile` of unit u: view group q of the unit's groups for G = u.cfg, detector range dr.
struct SfItem {
    int v0, cnt, cls, d0, Dt;
};

__device__ __forceinline__ SfItem sf_item(const Unit& u, int tile) {
    const int Dt = kSfConsumers / (u.lanes * u.cfg);
    const int n_dr = (u.D + Dt - 1) / Dt;
    const int q = tile / n_dr, dr = tile - q * n_dr;
    const Int2 grp = u.groups[q];
    return SfItem{grp.x, grp.y & 0xffff, grp.y >> 16, dr * Dt, Dt};
}

// Producer warp: the line of one of the item's extreme rays (first and last detector of each view),
// one per lane, in the compute frame.
struct SfEdge {
    float X0, Y0, sl;
    bool valid, flat;
};

__device__ __forceinline__ SfEdge sf_edge(const Unit& u, const SfItem& it) {
    const int lane = threadIdx.x & 31;
    SfEdge e{0.f, 0.f, 0.f, false, false};
    if (lane < 2 * it.cnt) {
        const int d = (lane & 1) ? min(it.d0 + it.Dt - 1, u.D - 1) : it.d0;
        const RayT r = u.rays[(long long)(it.v0 + (lane >> 1)) * u.D + d];
        e.X0 = it.cls ? (float)r.I0 + r.fy0 : (float)r.J0 + r.fx0;
        e.Y0 = it.cls ? (float)r.J0 + r.fx0 : (float)r.I0 + r.fy0;
        const float dX = it.cls ? r.dyh + r.dyl : r.dxh + r.dxl;
        const float dY = it.cls ? r.dxh + r.dxl : r.dyh + r.dyl;
        e.flat = fabsf(dY) <= 1e-6f * fabsf(dX);
        e.sl = e.flat ? 0.0f : dX / dY;
        e.valid = true;
    }
    return e;
}

// Band of slab s: the slab takes the samples whose texel row lies in [ylo, ylo + R), ylo = -2 + s R,
// and its buffer holds rows [ylo - 1, ylo + R] (one row of margin above: a sample that the previous
// slab left to this one may round to row ylo - 1 after re-basing).  Columns: those crossed by the
// extreme rays' lines over rows [ylo - 1, ylo + R + 1], clamped to the support, 2 columns of margin,
// the start aligned down to `align`.  [cs, ce) x [rs, re) is the part that exists in the packed image
// (rows and columns [-2, n]; columns rounded to whole 16-byte blocks).  Every lane returns the same band.
struct SfBand {
    int ylo, xc0, cs, ce, rs, re;
    bool empty, bad;
};

__device__ __forceinline__ SfBand sf_band(const SfEdge& e, int s, int R, int n, int wbox, int align) {
    SfBand b;
    b.ylo = -2 + s * R;
    float lo = 3.0e38f, hi = -3.0e38f;
    if (e.valid) {
        if (e.flat) {
            lo = -3.0f;
            hi = (float)n + 2.0f;
        } else {
            const float xa = fmaf((float)(b.ylo - 1) - e.Y0, e.sl, e.X0);
            const float xb = fmaf((float)(b.ylo + R + 1) - e.Y0, e.sl, e.X0);
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
    hi = fminf(hi, (float)n + 2.0f);
    b.empty = !(hi >= lo);
    if (b.empty) {
        lo = -3.0f;
        hi = -3.0f;
    }
    const int x_lo = (int)floorf(lo) - 2, x_hi = (int)ceilf(hi) + 2;
    b.xc0 = x_lo - (((x_lo % align) + align) % align);
    b.bad = x_hi - b.xc0 + 1 > wbox;
    b.cs = max(b.xc0, -2);
    b.ce = min(b.xc0 + wbox, n + 1);
    if (((b.ce - b.cs) & (align - 1)) != 0) ++b.ce;   // whole blocks: stays within the row and the band
    b.rs = max(b.ylo - 1, -2);
    b.re = min(b.ylo + R, n + 1);
    return b;
}

// Shared memory of the staged forward: full[4], empty[4] mbarriers, the abort flag, 4 headers of
// kSfHeaderInts ints, then `stages` buffers of (rmax + 1) x wbox texels (128-byte aligned each).
__host__ __device__ inline size_t sf_buffer_bytes(int rmax, int pitch, int qbytes) {
    return ((size_t)(rmax + 1) * pitch * qbytes + 127) / 128 * 128;
}
// Row pitch for bands of wbox texels: the band width itself.  (Offsetting consecutive rows by half a
// 128-byte line measured more shared-load bank conflicts on a 1024^2, 818-view image: 45 % of the
// wavefronts instead of 40 %, and one CTA per SM fewer in mixed plans.)
__host__ __device__ inline int sf_pitch(int wbox, int qbytes) {
    (void)qbytes;
    return wbox;
}
__host__ __device__ inline size_t sf_smem_bytes(int rmax, int wbox, int qbytes, int stages) {
    return 256 + (size_t)stages * sf_buffer_bytes(rmax, sf_pitch(wbox, qbytes), qbytes) + 128;   // + alignment slack
}

struct SfShared {
    uint64_t* full;
    uint64_t* empty;
    volatile int* abort_flag;
    int* hdr;
    unsigned char* bufs;
    size_t stride;
};

// Producer warp: takes work items (the device counter, or this CTA's one item) and streams each
// item's non-empty slabs into the ring; ends with a header of item -1.
template <typename T>
__device__ void sf_produce(const SfArgs& a, const SfShared& sh) {
    using Q = typename Quad<T>::type;
    constexpr int qb = (int)sizeof(Q);
    constexpr int align = qb == 8 ? 2 : 1;
    const int lane = threadIdx.x & 31;
    unsigned g = 0;   // slabs emitted so far (ring position)
    // Waits until buffer g % stages is free, then (lane 0) writes its header and announces `bytes`.
    auto claim = [&](int item, int s, int ylo, int xc0, int flags, uint32_t bytes) -> bool {
        const int buf = (int)(g % (unsigned)a.stages);
        bool ok = true;
        if (g >= (unsigned)a.stages && lane == 0)
            ok = mbar_wait_bounded(&sh.empty[buf], (g / (unsigned)a.stages - 1u) & 1u, a.spin_limit);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (lane == 0) {
            if (!ok) {
                record_device_error(a.err, RADON_ERR_TIMEOUT);
                *sh.abort_flag = 1;
                mbar_arrive(&sh.full[buf]);   // completes the phase without data: consumers see the abort
            } else {
                int* h = sh.hdr + buf * kSfHeaderInts;
                h[0] = item;
                h[1] = s;
                h[2] = ylo;
                h[3] = xc0;
                h[4] = flags;
                fence_proxy_async_shared();
                mbar_arrive_expect_tx(&sh.full[buf], bytes);
            }
        }
        __syncwarp();
        return ok;
    };
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1u);
        const int wi = (int)__shfl_sync(0xffffffffu, t, 0);
        if (wi >= a.n_work) {
            claim(-1, 0, 0, 0, 0, 0u);
            return;
        }
        const Work w = a.work[wi];
        const Unit& u = a.units[w.unit];
        const SfItem it = sf_item(u, w.tile);
        const SfEdge edge = sf_edge(u, it);
        const int R = u.R, n = u.n;
        const int n_slabs = (n + 3 + R - 1) / R;
        const long long P = sq_pitch(n);
        const unsigned char* frame = static_cast<const unsigned char*>(a.quads) +
                                     (size_t)(u.q_off + (it.cls ? sq_frame(n) : 0ll)) * qb;
        // the item's slabs run from its first to its last non-empty band; bands in between may be
        // empty (a view group across 90 degrees: edge rays near one side of the support reach it
        // at the top for some views and at the bottom for others) and are streamed without data
        int s = 0, s_last = n_slabs - 1;
        SfBand band = sf_band(edge, 0, R, n, a.wbox, align);
        while (band.empty && s + 1 < n_slabs) {
            ++s;
            band = sf_band(edge, s, R, n, a.wbox, align);
        }
        if (band.empty) {   // every ray misses the image: one slab without data, the sums stay 0
            if (!claim(wi, 0, band.ylo, band.xc0, kSfFirst | kSfLast | kSfNoData, 0u)) return;
            ++g;
            continue;
        }
        while (s_last > s && sf_band(edge, s_last, R, n, a.wbox, align).empty) --s_last;
        int flags = kSfFirst;
        for (;;) {
            if (s == s_last) flags |= kSfLast;
            if (band.empty) flags |= kSfNoData;
            if (lane == 0 && band.bad && !band.empty) record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
            const int rows = band.empty ? 0 : max(band.re - band.rs, 0), cols = max(band.ce - band.cs, 0);
            const uint32_t row_bytes = rows == 0 ? 0u : (uint32_t)cols * qb;
            if (!claim(wi, s, band.ylo, band.xc0, flags, (uint32_t)rows * row_bytes)) return;
            if (row_bytes != 0) {
                const int buf = (int)(g % (unsigned)a.stages);
                const uint32_t dst0 = smem_u32(sh.bufs + (size_t)buf * sh.stride);
                for (int r = band.rs + lane; r < band.re; r += 32)
                    bulk_load(dst0 + (uint32_t)(((r - band.ylo + 1) * a.pitch + (band.cs - band.xc0)) * qb),
                              frame + (size_t)((r + 2) * P + band.cs + 2) * qb, row_bytes, &sh.full[buf]);
            }
            ++g;
            if (flags & kSfLast) break;
            flags = 0;
            ++s;
            band = sf_band(edge, s, R, n, a.wbox, align);
        }
    }
}

// Consumer warps: thread t holds lane t % L of ray t / L of each item (views x detectors, detectors
// fastest); its partial sum over the item's slabs is joined with the ray's other lanes in a fixed
// shuffle tree and stored through the epilogue after the item's last slab.
template <typename T>
__device__ void sf_consume(const SfArgs& a, const SfShared& sh) {
    using Q = typename Quad<T>::type;
    constexpr unsigned qb = (unsigned)sizeof(Q);
    const int tid = threadIdx.x;
    const float M = 12582912.0f;          // 1.5 * 2^23: x + M rounds x to the nearest integer
    const unsigned magic = 0x4B400000u;   // the bit pattern of M
    const Unit* up = nullptr;
    int L = 1, sub = 0, R = 0, v = 0, d = 0, J0 = 0, I0 = 0, nk = 0, k = 0;
    bool active = false;
    float fX0 = 0.f, fY0 = 0.f, dXh = 0.f, dYh = 0.f, dXl = 0.f, dYl = 0.f, dX = 0.f, dY = 0.f, rdY = 0.f, acc = 0.f;
    for (unsigned g = 0;; ++g) {
        const int buf = (int)(g % (unsigned)a.stages);
        if (!mbar_wait_bounded(&sh.full[buf], (g / (unsigned)a.stages) & 1u, a.spin_limit)) {
            record_device_error(a.err, RADON_ERR_TIMEOUT);
            return;
        }
        if (*sh.abort_flag) return;
        const int* h = sh.hdr + buf * kSfHeaderInts;
        const int item = h[0];
        if (item < 0) return;
        const int ylo = h[2], xc0 = h[3], flags = h[4];
        if (flags & kSfFirst) {
            const Work w = a.work[item];
            up = &a.units[w.unit];
            const SfItem it = sf_item(*up, w.tile);
            L = up->lanes;
            R = up->R;
            const int ray = tid / L;
            sub = tid - ray * L;
            const int vl = ray / it.Dt, dl = ray - vl * it.Dt;
            v = it.v0 + vl;
            d = it.d0 + dl;
            active = vl < it.cnt && d < up->D;
            nk = 0;
            k = 0;
            acc = 0.0f;
            if (active) {
                const long long ridx = (long long)v * up->D + d;
                const RayT r = up->rays[ridx];
                nk = up->nks[ridx];
                if (it.cls == 0) {
                    J0 = r.J0; I0 = r.I0; fX0 = r.fx0; fY0 = r.fy0; dXh = r.dxh; dYh = r.dyh; dXl = r.dxl; dYl = r.dyl;
                } else {
                    J0 = r.I0; I0 = r.J0; fX0 = r.fy0; fY0 = r.fx0; dXh = r.dyh; dYh = r.dxh; dXl = r.dyl; dYl = r.dxl;
                }
                dX = dXh + dXl;
                dY = dYh + dYl;
                rdY = 1.0f / dY;   // inf for a ray along the rows: its slab count is then the rest
            }
        }
        int e = 0;   // samples of this slab, counted from k (the lanes of a ray agree after the min below)
        if (!(flags & kSfNoData) && k < nk) {
            const bool last = (flags & kSfLast) != 0;
            const float kf = (float)k;
            const float qX = kf * dXh, qY = kf * dYh;   // exact products
            const float QX = floorf(qX), QY = floorf(qY);
            const float sX = fmaf(kf, dXl, fX0 + (qX - QX));
            const float sY = fmaf(kf, dYl, fY0 + (qY - QY));
            const int JB = J0 + (int)QX - xc0;        // buffer-local integer base of sample k
            const int IB = I0 + (int)QY - (ylo - 1);   // (buffer row 0 = texel row ylo - 1)
            // this slab's samples: texel row below ylo + R, i.e. buffer row <= R
            const float ylim_m = last ? 3.0e38f : (float)(R + 1 - IB) - 0.5f;
            const float sYm = sY - 0.5f;
            const int kleft = nk - k;
            // the ray's next sample may lie in a later slab (rays entering through a side): nothing here
            if (sYm < ylim_m) {
                // c = this slab's samples: the first j with row j at or past the limit (rows grow with j),
                // from a quotient corrected in the exact arithmetic of the test, the same on every lane
                int c = kleft;
                if (!last) {
                    const float est = ceilf((ylim_m - sYm) * rdY);
                    c = est < (float)kleft ? max((int)est, 1) : kleft;
                    while (c > 1 && fmaf((float)(c - 1), dY, sYm) >= ylim_m) --c;
                    while (c < kleft && fmaf((float)c, dY, sYm) < ylim_m) ++c;
                }
                // every sample this slab takes stays inside the buffer (the extreme rays' lines enclose
                // the item's rays); checked per ray, so no access leaves it
                // (rows: the count keeps a non-last slab's samples at buffer row <= R; the last slab's
                // final sample is tested in the loop's own arithmetic)
                const float xa = (float)JB + sX, ya = (float)IB + sY;
                const float xb = fmaf((float)(c - 1), dX, xa);
                if (fminf(xa, xb) < 0.25f || fmaxf(xa, xb) > (float)a.wbox - 1.25f || ya < 0.5f ||
                    (last && fmaf((float)(c - 1), dY, sYm) >= (float)(R + 1 - IB) - 0.5f)) {
                    record_device_error(a.err, RADON_ERR_DEVICE_BOUNDS);
                    e = kleft;
                } else {
                    const float sXm = sX - 0.5f;
                    const unsigned rowb = (unsigned)a.pitch * qb;
                    // shared address of texel (row, col) = buffer + qb (row pitch + col): the magic-biased
                    // bit patterns of the floors enter modulo 2^32, so the biases cancel exactly
                    const unsigned base = smem_u32(sh.bufs + (size_t)buf * sh.stride) +
                                          qb * (unsigned)(IB * a.pitch + JB) - magic * (rowb + qb);
                    auto sample = [&](float kk) {
                        const float fym = fmaf(kk, dY, sYm), fxm = fmaf(kk, dX, sXm);
                        const float tx = fxm + M, ty = fym + M;
                        float t[4];
                        sq_load<T>(__float_as_uint(ty) * rowb + __float_as_uint(tx) * qb + base, t);
                        const float ax = (fxm - (tx - M)) + 0.5f, ay = (fym - (ty - M)) + 0.5f;   // in [0, 1]
                        const float top = fmaf(ax, t[1] - t[0], t[0]), bot = fmaf(ax, t[3] - t[2], t[2]);
                        acc += fmaf(ay, bot - top, top);
                    };
                    const float step = (float)L;
                    int j = sub;
                    float kk = (float)sub;
                    for (; j + L < c; j += 2 * L, kk += 2.0f * step) {
                        sample(kk);
                        sample(kk + step);
                    }
                    if (j < c) sample(kk);
                    e = c;
                }
            }
        }
        k += e;   // the same on every lane of a ray
        mbar_arrive(&sh.empty[buf]);   // this thread's reads of the buffer are done
        if (flags & kSfLast) {
            float y = acc;
            if (L > 1) {
                y += __shfl_xor_sync(0xffffffffu, y, 1);
                y += __shfl_xor_sync(0xffffffffu, y, 2);
            }
            if (active && sub == 0) {
                const long long idx = (long long)v * up->D + d;
                static_cast<T*>(up->out)[idx] = from_f32<T>(epilogue_value<T>(a.ep, up->h * y, idx));
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSfThreads, 3) staged_forward_kernel(const SfArgs a) {
    using Q = typename Quad<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    SfShared sh;
    sh.full = reinterpret_cast<uint64_t*>(smem);
    sh.empty = reinterpret_cast<uint64_t*>(smem + 32);
    sh.abort_flag = reinterpret_cast<volatile int*>(smem + 64);
    sh.hdr = reinterpret_cast<int*>(smem + 128);
    sh.bufs = smem + 256;
    sh.stride = sf_buffer_bytes(a.rmax, a.pitch, (int)sizeof(Q));
    const int tid = threadIdx.x;
    if (tid < a.stages) {
        mbar_init(&sh.full[tid], 1);
        mbar_init(&sh.empty[tid], kSfConsumers);
    }
    if (tid == 0) *sh.abort_flag = 0;
    fence_mbar_init();
    __syncthreads();
    if ((tid >> 5) == kSfConsumerWarps)
        sf_produce<T>(a, sh);
    else
        sf_consume<T>(a, sh);
}

// One thread per quad texel of every unit (both frames); `prefix[u]` = first texel of unit u.
template <typename T>
__global__ void __launch_bounds__(256) sq_pack_kernel(const Unit* __restrict__ units, const long long* __restrict__ prefix,
                                                      int n_units, long long total, typename Quad<T>::type* __restrict__ quads) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += stride) {
        int lo = 0, hi = n_units - 1;   // last unit with prefix <= gi
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= gi) lo = mid;
            else hi = mid - 1;
        }
        const Unit& u = units[lo];
        quads[gi] = sq_texel<T>(static_cast<const T*>(u.in), u.n, gi - prefix[lo]);
    }
}

// The same for one image (a batch-1 call).
template <typename T>
__global__ void __launch_bounds__(256) sq_pack_single_kernel(const T* __restrict__ x, int n,
                                                             typename Quad<T>::type* __restrict__ quads) {
    const long long total = 2 * sq_frame(n);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += stride)
        quads[gi] = sq_texel<T>(x, n, gi);
}

}  // namespace radon
