/*
 * FP64 CPU oracle for the discrete Radon transform and its exact adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library: its own geometry, its own sample enumeration, its own
 * interpolation.  It is deliberately plain and slow: no tiling, no clipping
 * algebra, no fusion.
 *
 * What it computes.  The paper names the operators and their geometry
 * parameters (Section 3.1.1: angles, det_count, det_spacing; Section 3.1.2:
 * source_distance, det_distance, a flat detector) but not the discretisation;
 * the reading used throughout is fixed-step bilinear sampling along each ray:
 *
 *   Image x[b][i][j] (row i, column j), pixel centre (j - (N-1)/2, i - (N-1)/2).
 *   Sinogram y[b][v][d], V views, D detector bins of spacing ds, step h.
 *
 *   Ray (v, d)  -- Section 3.1.1 (parallel beam) and 3.1.2 (fan beam):
 *     n = (cos t, sin t), u = (-sin t, cos t), s_d = (d - (D-1)/2) * ds.
 *     parallel: origin m = s_d n, direction u.
 *     fan:      source c = -S u, detector bin q = Ddet u + s_d n (flat detector
 *               at distance Ddet from the centre), direction r = (q-c)/|q-c|,
 *               origin m = c - (c.r) r (foot of the perpendicular from the
 *               rotation centre).
 *   Samples  p_k = m + k h u for every integer k with p_k strictly inside the
 *            box (-(N+1)/2, (N+1)/2)^2 (outside it every bilinear weight that
 *            lands on a pixel is zero).  The oracle scans a generous k range and
 *            tests membership; it does no clipping arithmetic.
 *   Value    bilinear interpolation of x at p_k, pixels outside [0,N)^2 read 0.
 *   Forward  y[b][v][d] = h * sum_k value(p_k), a fixed-step approximation of
 *            the line integral of the bilinear image (Section 3.1.1).
 *   Adjoint  literal scatter: every sample adds h*y[b][v][d]*weight to each of
 *            its four pixels (the transpose of the forward, Section 3.1.1
 *            "backprojection", read as the exact discrete adjoint).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;                  /* image side N */
    int n_angles;           /* V */
    const double *angles;   /* theta_v, radians */
    int det_count;          /* D */
    double det_spacing;     /* ds */
    double step;            /* h */
    int fan;                /* 0: parallel beam, 1: fan beam */
    double source_distance; /* S (fan) */
    double det_distance;    /* Ddet (fan) */
} oracle_geometry;

/* Ray origin m and unit direction u of ray (v, d) (Sections 3.1.1, 3.1.2). */
void oracle_ray(const oracle_geometry *g, int v, int d, double m[2], double u[2])
{
    double th = g->angles[v];
    double nx = cos(th), ny = sin(th);
    double ux = -sin(th), uy = cos(th);
    double s = ((double)d - 0.5 * (double)(g->det_count - 1)) * g->det_spacing;
    if (!g->fan) {
        m[0] = s * nx;
        m[1] = s * ny;
        u[0] = ux;
        u[1] = uy;
        return;
    }
    double cx = -g->source_distance * ux, cy = -g->source_distance * uy;   /* source */
    double qx = g->det_distance * ux + s * nx, qy = g->det_distance * uy + s * ny; /* bin */
    double rx = qx - cx, ry = qy - cy;
    double len = sqrt(rx * rx + ry * ry);
    rx /= len;
    ry /= len;
    double cr = cx * rx + cy * ry;
    m[0] = cx - cr * rx;
    m[1] = cy - cr * ry;
    u[0] = rx;
    u[1] = ry;
}

/* Largest |k| worth scanning: |p_k| >= |k h| - |m| and the box has half-diagonal (N+1)/sqrt 2. */
static long k_scan_limit(const oracle_geometry *g)
{
    return (long)ceil((double)g->n / g->step) + 2;
}

/* Sample position p_k and whether it lies strictly inside the support box. */
static int sample_at(const oracle_geometry *g, const double m[2], const double u[2], long k, double p[2])
{
    double t = (double)k * g->step;
    double half = 0.5 * (double)(g->n + 1);
    p[0] = m[0] + t * u[0];
    p[1] = m[1] + t * u[1];
    return fabs(p[0]) < half && fabs(p[1]) < half;
}

/* Bilinear interpolation of one image at p (pixel units, image-centred). */
static double bilinear(const double *img, int n, const double p[2])
{
    double fx = p[0] + 0.5 * (double)(n - 1);
    double fy = p[1] + 0.5 * (double)(n - 1);
    double j0 = floor(fx), i0 = floor(fy);
    double a = fx - j0, b = fy - i0;
    long j = (long)j0, i = (long)i0;
    double v = 0.0;
    for (int di = 0; di <= 1; ++di) {
        for (int dj = 0; dj <= 1; ++dj) {
            long ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
            double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);
            v += w * img[ii * n + jj];
        }
    }
    return v;
}

/* Transpose of bilinear(): add val * weight into the four pixels around p. */
static void bilinear_scatter(double *img, int n, const double p[2], double val)
{
    double fx = p[0] + 0.5 * (double)(n - 1);
    double fy = p[1] + 0.5 * (double)(n - 1);
    double j0 = floor(fx), i0 = floor(fy);
    double a = fx - j0, b = fy - i0;
    long j = (long)j0, i = (long)i0;
    for (int di = 0; di <= 1; ++di) {
        for (int dj = 0; dj <= 1; ++dj) {
            long ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
            double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);
            img[ii * n + jj] += w * val;
        }
    }
}

/* Number of samples of every ray of one image: the throughput unit. */
int64_t oracle_sample_count(const oracle_geometry *g)
{
    int64_t total = 0;
    long kmax = k_scan_limit(g);
    for (int v = 0; v < g->n_angles; ++v) {
        for (int d = 0; d < g->det_count; ++d) {
            double m[2], u[2], p[2];
            oracle_ray(g, v, d, m, u);
            for (long k = -kmax; k <= kmax; ++k) total += sample_at(g, m, u, k, p);
        }
    }
    return total;
}

/* Per-ray sample counts, [V][D] (for tests of the clipping). */
void oracle_ray_sample_counts(const oracle_geometry *g, int64_t *counts)
{
    long kmax = k_scan_limit(g);
    for (int v = 0; v < g->n_angles; ++v) {
        for (int d = 0; d < g->det_count; ++d) {
            double m[2], u[2], p[2];
            int64_t c = 0;
            oracle_ray(g, v, d, m, u);
            for (long k = -kmax; k <= kmax; ++k) c += sample_at(g, m, u, k, p);
            counts[(int64_t)v * g->det_count + d] = c;
        }
    }
}

/* Forward projection: sino[b][v][d] = h * sum_k bilinear(img[b], p_k). */
void oracle_forward(const oracle_geometry *g, const double *img, double *sino, int batch)
{
    const int64_t npix = (int64_t)g->n * g->n;
    const int64_t nsino = (int64_t)g->n_angles * g->det_count;
    long kmax = k_scan_limit(g);
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int b = 0; b < batch; ++b) {
        for (int v = 0; v < g->n_angles; ++v) {
            const double *x = img + b * npix;
            for (int d = 0; d < g->det_count; ++d) {
                double m[2], u[2], p[2];
                double acc = 0.0;
                oracle_ray(g, v, d, m, u);
                for (long k = -kmax; k <= kmax; ++k) {
                    if (sample_at(g, m, u, k, p)) acc += bilinear(x, g->n, p);
                }
                sino[b * nsino + (int64_t)v * g->det_count + d] = g->step * acc;
            }
        }
    }
}

/* Exact adjoint by literal scatter: img[b] = sum_{v,d,k} h*sino[b][v][d]*weights(p_k). */
void oracle_adjoint(const oracle_geometry *g, const double *sino, double *img, int batch)
{
    const int64_t npix = (int64_t)g->n * g->n;
    const int64_t nsino = (int64_t)g->n_angles * g->det_count;
    long kmax = k_scan_limit(g);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < batch; ++b) {
        double *x = img + b * npix;
        memset(x, 0, sizeof(double) * (size_t)npix);
        for (int v = 0; v < g->n_angles; ++v) {
            for (int d = 0; d < g->det_count; ++d) {
                double m[2], u[2], p[2];
                double val = g->step * sino[b * nsino + (int64_t)v * g->det_count + d];
                oracle_ray(g, v, d, m, u);
                for (long k = -kmax; k <= kmax; ++k) {
                    if (sample_at(g, m, u, k, p)) bilinear_scatter(x, g->n, p, val);
                }
            }
        }
    }
}

/* Number of OpenMP threads the oracle runs on (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
