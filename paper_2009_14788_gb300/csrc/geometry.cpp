// FP64 geometry tables (host).  Everything here runs once per geometry; kernels only read the
// FP32 tables it produces.
//
// Ray construction follows the parallel-beam (Section 3.1.1) and flat-detector fan-beam
// (Section 3.1.2) set-ups: view angle t, n = (cos t, sin t), u = (-sin t, cos t), bin offset
// s_d = (d - (D-1)/2) ds.  Parallel: origin s_d n, direction u.  Fan: source -S u, bin
// Ddet u + s_d n, unit direction r from source to bin, origin = foot of the perpendicular from
// the rotation centre onto the ray.  Samples p_k = m + k h r, k integer, strictly inside the
// support box (-(N+1)/2, (N+1)/2)^2.
#include <algorithm>
#include <cmath>
#include <limits>

#include "radon_internal.h"

namespace radon {

namespace {

struct Ray64 {
    double mx, my, ux, uy;
};

Ray64 make_ray(const radon_geometry* g, int v, int d) {
    const double th = g->angles[v];
    const double c = std::cos(th), s = std::sin(th);
    const double nx = c, ny = s, ux = -s, uy = c;
    const double sd = ((double)d - 0.5 * (double)(g->D - 1)) * g->ds;
    Ray64 r;
    if (!g->fan) {
        r.mx = sd * nx;
        r.my = sd * ny;
        r.ux = ux;
        r.uy = uy;
        return r;
    }
    const double srcx = -g->S * ux, srcy = -g->S * uy;
    const double qx = g->Ddet * ux + sd * nx, qy = g->Ddet * uy + sd * ny;
    double ex = qx - srcx, ey = qy - srcy;
    const double len = std::sqrt(ex * ex + ey * ey);
    ex /= len;
    ey /= len;
    const double along = srcx * ex + srcy * ey;   // source coordinate along the ray
    r.mx = srcx - along * ex;
    r.my = srcy - along * ey;
    r.ux = ex;
    r.uy = ey;
    return r;
}

// Membership of sample k, evaluated exactly as the definition states it: t = k h, p = m + t u.
bool inside(const radon_geometry* g, const Ray64& r, long k) {
    const double half = 0.5 * (double)(g->n + 1);
    const double t = (double)k * g->h;
    const double px = r.mx + t * r.ux, py = r.my + t * r.uy;
    return std::fabs(px) < half && std::fabs(py) < half;
}

// [klo, khi] of the samples inside the open box: slab clipping, then an exact re-check so the
// result agrees with the membership test sample by sample.  Returns false if empty.
bool k_range(const radon_geometry* g, const Ray64& r, long* klo, long* khi) {
    const double half = 0.5 * (double)(g->n + 1);
    double lo = -std::numeric_limits<double>::infinity(), hi = std::numeric_limits<double>::infinity();
    const double m[2] = {r.mx, r.my}, u[2] = {r.ux, r.uy};
    for (int a = 0; a < 2; ++a) {
        if (u[a] != 0.0) {
            double t1 = (-half - m[a]) / (g->h * u[a]);
            double t2 = (half - m[a]) / (g->h * u[a]);
            if (t1 > t2) std::swap(t1, t2);
            lo = std::max(lo, t1);
            hi = std::min(hi, t2);
        } else if (std::fabs(m[a]) >= half) {
            return false;
        }
    }
    if (!(lo < hi)) return false;
    long a = (long)std::floor(lo) + 1, b = (long)std::ceil(hi) - 1;
    // Rounding of m + t u is monotone in t, so the FP64 inside set is an interval of integers.
    // Move both ends onto its exact boundary.  Shrinking can take many steps for a ray that runs
    // along a box edge (every sample sits within rounding of the edge); growing takes at most a
    // few because the slab bounds are exact up to rounding.
    while (a <= b && !inside(g, r, a)) ++a;
    while (b >= a && !inside(g, r, b)) --b;
    if (a > b) return false;
    for (int it = 0; it < 8 && inside(g, r, a - 1); ++it) --a;
    for (int it = 0; it < 8 && inside(g, r, b + 1); ++it) ++b;
    if (a > b) return false;
    *klo = a;
    *khi = b;
    return true;
}

// Round v to `bits` significant bits (toward nearest).
double round_bits(double v, int bits) {
    if (v == 0.0) return 0.0;
    int e = 0;
    const double m = std::frexp(v, &e);   // v = m 2^e, 0.5 <= |m| < 1
    return std::ldexp(std::nearbyint(std::ldexp(m, bits)), e - bits);
}

// Integer base and fraction in [0, 1) of a coordinate, the fraction rounded to FP32.
void split_coord(double p, int* base, float* frac) {
    double b = std::floor(p);
    float f = (float)(p - b);
    if (f >= 1.0f) {   // the FP32 rounding of a fraction just below 1
        b += 1.0;
        f = 0.0f;
    }
    *base = (int)b;
    *frac = f;
}

}  // namespace

radon_status build_geometry(radon_geometry* g) {
    const int V = g->V, D = g->D;
    const double c0 = 0.5 * (double)(g->n - 1);
    g->h_ray.assign((size_t)V * D, RayT{0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f});
    g->h_nk.assign((size_t)V * D, 0);
    g->h_view.assign((size_t)V, ViewF{});
    int64_t total = 0;
    int max_nk = 0;
    for (int v = 0; v < V; ++v) {
        const double th = g->angles[v];
        const double nx = std::cos(th), ny = std::sin(th), ux = -std::sin(th), uy = std::cos(th);
        const int major = std::fabs(uy) >= std::fabs(ux) ? 0 : 1;
        // Projective detector map in centred coordinates P:
        //   parallel  t = (n.P)/ds + (D-1)/2
        //   fan       t = [((S+Ddet)/ds) n.P + ((D-1)/2)(S + u.P)] / (S + u.P)
        // then shifted to index coordinates (x = P.x + c0, y = P.y + c0).
        double Ax, Ay, A0, Bx, By, B0;
        const double half_d = 0.5 * (double)(D - 1);
        if (!g->fan) {
            Ax = nx / g->ds;
            Ay = ny / g->ds;
            A0 = half_d;
            Bx = 0.0;
            By = 0.0;
            B0 = 1.0;
        } else {
            const double mag = (g->S + g->Ddet) / g->ds;
            Ax = mag * nx + half_d * ux;
            Ay = mag * ny + half_d * uy;
            A0 = half_d * g->S;
            Bx = ux;
            By = uy;
            B0 = g->S;
        }
        ViewF& vf = g->h_view[v];
        vf.ax = (float)Ax;
        vf.ay = (float)Ay;
        vf.a0 = (float)(A0 - c0 * (Ax + Ay));
        vf.bx = (float)Bx;
        vf.by = (float)By;
        vf.b0 = (float)(B0 - c0 * (Bx + By));
        vf.major = major;
        vf.pad = 0;
        for (int d = 0; d < D; ++d) {
            const Ray64 r = make_ray(g, v, d);
            long klo = 0, khi = -1;
            const size_t idx = (size_t)v * D + d;
            // A ray that misses the image keeps its line (sample 0 = the foot point) with no samples:
            // the tiled forward bounds its working band with the lines of its extreme rays.
            const bool hit = k_range(g, r, &klo, &khi);
            if (!hit) {
                klo = 0;
                khi = 0;
            }
            const int nk = hit ? (int)(khi - klo + 1) : 0;
            double sx = g->h * r.ux, sy = g->h * r.uy;
            long kstart = klo;
            const bool flip = major == 0 ? (sy < 0.0) : (sx < 0.0);
            if (flip) {
                kstart = khi;
                sx = -sx;
                sy = -sy;
            }
            const double t = (double)kstart * g->h;
            const double px = r.mx + t * r.ux + c0, py = r.my + t * r.uy + c0;
            RayT& rt = g->h_ray[idx];
            split_coord(px, &rt.J0, &rt.fx0);
            split_coord(py, &rt.I0, &rt.fy0);
            // k' * dxh exact in FP32 for -M <= k' < nk + M: dxh keeps 24 - bits(nk + M) significant bits.
            // The margin M covers the adjoint's reference sample, the one nearest a 16-pixel tile's
            // centre, which may sit up to (tile half-diagonal + support) / h samples past a ray end.
            const long margin = kSplitMarginPx * (long)std::ceil(1.0 / g->h) + 8;
            int kbits = 1;
            while (kbits < 24 && ((long)1 << kbits) < (long)nk + margin) ++kbits;
            const int hbits = std::max(1, 24 - kbits);
            const double hx = round_bits(sx, hbits), hy = round_bits(sy, hbits);
            rt.dxh = (float)hx;
            rt.dyh = (float)hy;
            rt.dxl = (float)(sx - hx);
            rt.dyl = (float)(sy - hy);
            g->h_nk[idx] = nk;
            total += nk;
            if (nk > max_nk) max_nk = nk;
        }
    }
    g->samples = total;
    g->max_nk = max_nk;
    g->bwd_window = backward_window_width(g, 16);
    // The tiled forward gives each 8-lane phase of its 16-byte shared loads two neighbouring views x
    // four detectors when the rays of consecutive views stay within 5 pixels of each other inside the
    // image ((n / 2) |theta_{v+1} - theta_v| <= 5): their texels then fall in fewer bank groups than
    // eight detectors of one view.  With wider view steps the pair spreads over more columns and one
    // view per phase is faster (measured over view counts 60 to 720, parallel and fan beam).
    double gap = 0.0;
    for (int v = 0; v + 1 < V; ++v) gap = std::max(gap, std::fabs(g->angles[v + 1] - g->angles[v]));
    g->fwd_pair_views = V >= 2 && 0.5 * g->n * gap <= 5.0 ? 1 : 0;
    // Groups of up to G consecutive views of one orientation class (the tiled forward's CTAs):
    // entry = (first view, count | class << 16), for G = 1, 2, 4, 8.
    g->h_groups.clear();
    for (int gi = 0; gi < 4; ++gi) {
        const int G = 1 << gi;
        g->group_offset[gi] = (int)g->h_groups.size();
        int v = 0;
        while (v < V) {
            const int cls = g->h_view[v].major;
            int cnt = 1;
            while (cnt < G && v + cnt < V && g->h_view[v + cnt].major == cls) ++cnt;
            g->h_groups.push_back(Int2{v, cnt | (cls << 16)});
            v += cnt;
        }
        g->group_count[gi] = (int)g->h_groups.size() - g->group_offset[gi];
    }
    return RADON_OK;
}

namespace {

double view_t(const ViewF& vf, double x, double y) {
    return ((double)vf.ax * x + (double)vf.ay * y + (double)vf.a0) / ((double)vf.bx * x + (double)vf.by * y + (double)vf.b0);
}

// Detector window [floor(tmin - r - 0.01), floor(tmax + r)] of one tile and view, as the tiled adjoint
// computes it (the kernel uses FP32; the caller adds slack).
int tile_window(const radon_geometry* g, const ViewF& vf, int ti, int tj, int tile) {
    const double x0 = tj, x1 = std::min(tj + tile - 1, g->n - 1), y0 = ti, y1 = std::min(ti + tile - 1, g->n - 1);
    const double ts[4] = {view_t(vf, x0, y0), view_t(vf, x1, y0), view_t(vf, x0, y1), view_t(vf, x1, y1)};
    const double tmin = std::min(std::min(ts[0], ts[1]), std::min(ts[2], ts[3]));
    const double tmax = std::max(std::max(ts[0], ts[1]), std::max(ts[2], ts[3]));
    double r;
    if (vf.bx == 0.0f && vf.by == 0.0f) {
        r = (std::fabs((double)vf.ax) + std::fabs((double)vf.ay)) / (double)vf.b0;
    } else {
        r = 0.0;
        for (int c = 0; c < 4; ++c) {
            const double cx = (c & 1) ? x1 : x0, cy = (c & 2) ? y1 : y0;
            const double s[4] = {view_t(vf, cx - 1, cy - 1), view_t(vf, cx + 1, cy - 1), view_t(vf, cx - 1, cy + 1),
                                 view_t(vf, cx + 1, cy + 1)};
            const double mx = std::max(std::max(s[0], s[1]), std::max(s[2], s[3]));
            const double mn = std::min(std::min(s[0], s[1]), std::min(s[2], s[3]));
            r = std::max(r, 0.5 * (mx - mn));
        }
        r = r * 1.05 + 0.02;
    }
    r += 0.01;
    const double lo = std::floor(tmin - r - 0.01), hi = std::floor(tmax + r);
    return (int)(hi - lo) + 1;
}

}  // namespace

int backward_window_width(const radon_geometry* g, int tile) {
    const int tiles = (g->n + tile - 1) / tile;
    const bool all = (double)tiles * tiles * g->V <= 2e7;
    int w = 0;
    for (int v = 0; v < g->V; ++v) {
        const ViewF& vf = g->h_view[v];
        for (int a = 0; a < tiles; ++a) {
            for (int b = 0; b < tiles; ++b) {
                // very large geometries: boundary tiles only (the projected width peaks nearest the
                // source, i.e. on the image boundary) plus a 10% margin below
                if (!all && a != 0 && a != tiles - 1 && b != 0 && b != tiles - 1) continue;
                w = std::max(w, tile_window(g, vf, a * tile, b * tile, tile));
            }
        }
    }
    if (!all) w = w + w / 10 + 1;
    return w;
}

}  // namespace radon

namespace radon {

// Widest band of the tiled forward, in compute-frame columns: for every CTA (view group x detector
// range) and slab, the columns between the lines of the CTA's extreme rays over the slab's buffer
// rows (+-1 row), clamped to the support, with 2 columns of margin on each side -- the formula the
// kernel evaluates in FP32 (the launcher adds slack for the difference).
int forward_band_width(radon_geometry* g, int G, int Dt, int R) {
    const long long key = ((long long)G << 40) | ((long long)Dt << 20) | (long long)R;
    std::lock_guard<std::mutex> lock(g->band_mu);
    auto it = g->band_width.find(key);
    if (it != g->band_width.end()) return it->second;
    int gi = 0;
    while ((1 << gi) < G) ++gi;
    const int n_slabs = (g->n + 4 + R - 1) / R;
    const int n_dr = (g->D + Dt - 1) / Dt;
    int maxw = 0;
    for (int q = 0; q < g->group_count[gi]; ++q) {
        const Int2 grp = g->h_groups[g->group_offset[gi] + q];
        const int v0 = grp.x, cnt = grp.y & 0xffff, cls = grp.y >> 16;
        for (int dr = 0; dr < n_dr; ++dr) {
            const int d0 = dr * Dt, d1 = std::min(d0 + Dt - 1, g->D - 1);
            for (int s = 0; s < n_slabs; ++s) {
                const double ylo = -4.0 + s * R, yhi = ylo + R + 1.0;
                double xmin = 1e300, xmax = -1e300;
                for (int vl = 0; vl < cnt; ++vl) {
                    for (int e = 0; e < 2; ++e) {
                        const RayT& r = g->h_ray[(size_t)(v0 + vl) * g->D + (e ? d1 : d0)];
                        const double X0 = cls ? (double)r.I0 + r.fy0 : (double)r.J0 + r.fx0;
                        const double Y0 = cls ? (double)r.J0 + r.fx0 : (double)r.I0 + r.fy0;
                        const double dX = cls ? (double)r.dyh + r.dyl : (double)r.dxh + r.dxl;
                        const double dY = cls ? (double)r.dxh + r.dxl : (double)r.dyh + r.dyl;
                        if (std::fabs(dY) <= 1e-6 * std::fabs(dX)) {
                            xmin = std::min(xmin, -3.0);
                            xmax = std::max(xmax, g->n + 2.0);
                        } else {
                            const double sl = dX / dY;
                            const double xa = X0 + (ylo - 1.0 - Y0) * sl, xb = X0 + (yhi + 1.0 - Y0) * sl;
                            xmin = std::min(xmin, std::min(xa, xb));
                            xmax = std::max(xmax, std::max(xa, xb));
                        }
                    }
                }
                xmin = std::max(xmin, -3.0);
                xmax = std::min(xmax, g->n + 2.0);
                if (xmax < xmin) continue;
                const int w = (int)(std::ceil(xmax) + 2 - (std::floor(xmin) - 2)) + 1;
                maxw = std::max(maxw, w);
            }
        }
    }
    g->band_width[key] = maxw;
    return maxw;
}

}  // namespace radon
