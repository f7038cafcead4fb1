/*
 * radon.h -- C ABI of libradon: the discrete Radon transform (forward projection)
 * and its exact adjoint (backprojection) on one NVIDIA GB300 (sm_103a) GPU.
 *
 * The operations follow TorchRadon's statement of the problem (Ronchetti 2020):
 *   - Section 3.1.1: parallel-beam projection with a set of angles, a detector of
 *     det_count bins of det_spacing (defaults: det_count = image size, spacing 1).
 *   - Section 3.1.2: fan-beam projection with a point source at source_distance
 *     from the centre and a flat detector at det_distance (default: equal to
 *     source_distance); default det_spacing is the smallest one whose bins cover
 *     the magnified image, (S + Ddet) / S * N / det_count (the worked example
 *     S = Ddet = 512, N = det_count = 512 gives 2.0).
 *   - Section 3.1.1 / 3.1.2 "forward" and "backprojection", batched over any
 *     number of images (Section 4.1), 16-bit storage with 32-bit arithmetic
 *     (Section 3.3).
 *
 * The discretisation (the paper does not spell it out) is fixed-step bilinear
 * ray sampling.  Image x[b][i][j] (row i, column j) has its pixel centre at
 * (j - (N-1)/2, i - (N-1)/2).  View v has n = (cos t, sin t), u = (-sin t, cos t);
 * detector bin d sits at s_d = (d - (D-1)/2) * det_spacing.  Ray (v, d):
 *   parallel: origin m = s_d n, direction u;
 *   fan:      source c = -S u, bin q = Ddet u + s_d n, direction r = (q - c)/|q - c|,
 *             origin m = the point of the ray closest to the rotation centre.
 * Samples p_k = m + k h r for every integer k with p_k strictly inside the box
 * (-(N+1)/2, (N+1)/2)^2; each sample is the bilinear interpolation of x (zero
 * outside the image).  Forward: y[b][v][d] = h * sum_k sample.  Backward: the
 * exact transpose, x[b] = h * sum_{v,d,k} y[b][v][d] * (bilinear weights of p_k).
 *
 * Conventions for every call below:
 *   - Memory: device pointers, C-contiguous.  Image [batch][N][N], sinogram
 *     [batch][n_angles][det_count], both of the same radon_dtype.  The caller
 *     owns every buffer passed in; outputs are overwritten, never accumulated.
 *     Arithmetic is FP32 for every storage type; 16-bit outputs are rounded to
 *     nearest even.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     radon_forward / radon_backward / radon_batch_plan_launch allocate nothing,
 *     never synchronise and can be captured in a CUDA graph.  Geometry and plan
 *     creation allocate and synchronise and must not run during capture.
 *   - Devices: a geometry belongs to the device that was current at creation;
 *     launching it with another device current is RADON_ERR_INVALID_ARG.
 *   - Errors: every call returns a radon_status and never throws or exits.
 *     Argument errors are detected on the host before any launch.  Kernels that
 *     wait on asynchronous copies bound every wait; on expiry they record
 *     RADON_ERR_TIMEOUT in a device error word that radon_get_device_error reads.
 *     radon_last_error_message gives a thread-local description of the last
 *     failure.
 */
#ifndef RADON_H
#define RADON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RADON_ABI_VERSION 2

#if defined(__GNUC__)
#define RADON_API __attribute__((visibility("default")))
#else
#define RADON_API
#endif

typedef enum {
    RADON_OK = 0,
    RADON_ERR_INVALID_ARG = 1,   /* bad pointer, size, dtype, geometry handle or device */
    RADON_ERR_UNSUPPORTED = 2,   /* valid request this build cannot serve (e.g. tile config) */
    RADON_ERR_OOM = 3,           /* device or host allocation failed (create calls only) */
    RADON_ERR_CUDA = 4,          /* a CUDA runtime / driver call failed; see the message */
    RADON_ERR_TIMEOUT = 5,       /* a kernel's bounded wait expired (device error word) */
    RADON_ERR_DEVICE_BOUNDS = 6  /* a kernel's own bounds check fired (device error word) */
} radon_status;

typedef enum {
    RADON_F32 = 0,   /* float32 storage */
    RADON_F16 = 1,   /* IEEE half storage, FP32 arithmetic */
    RADON_BF16 = 2   /* bfloat16 storage, FP32 arithmetic */
} radon_dtype;

typedef enum {
    RADON_ALGO_AUTO = 0,   /* the tuned kernels (what radon_forward / radon_backward run) */
    RADON_ALGO_PLAIN = 1,  /* one thread per ray (forward) / per pixel (backward), global loads */
    RADON_ALGO_TILED = 2   /* TMA-staged shared-memory tiles, explicit parameters below */
} radon_algo;

/* Opaque geometry: FP64-built ray tables uploaded to the device, owned by the library. */
typedef struct radon_geometry radon_geometry;

/*
 * Parallel beam (Section 3.1.1).
 *   n           image side N (>= 1, <= 8192)
 *   angles      host array of n_angles view angles in radians (read during the call only)
 *   det_count   detector bins D; <= 0 selects N
 *   det_spacing bin spacing in pixels; <= 0 selects 1.0
 *   step        sampling step h along each ray in pixels; <= 0 selects 1.0
 *   out         receives the new geometry (NULL on failure)
 * Allocates host and device memory; synchronises the current device.
 */
RADON_API radon_status radon_geometry_create_parallel(int n, const double* angles, int n_angles, int det_count,
                                            double det_spacing, double step, radon_geometry** out);

/*
 * Fan beam with a flat detector (Section 3.1.2).
 *   source_distance  S > 0, source to rotation centre, pixels
 *   det_distance     rotation centre to detector; <= 0 selects S
 *   det_count        <= 0 selects N
 *   det_spacing      <= 0 selects (S + Ddet) / S * N / det_count
 *   other arguments as for radon_geometry_create_parallel.
 */
RADON_API radon_status radon_geometry_create_fanbeam(int n, const double* angles, int n_angles, double source_distance,
                                           double det_distance, int det_count, double det_spacing, double step,
                                           radon_geometry** out);

/*
 * General constructor.  `host_only` != 0 builds the FP64 tables on the host without touching
 * any GPU (for inspection and tests on machines without one); such a geometry answers
 * radon_geometry_get_info / radon_geometry_sample_count / radon_geometry_copy_rays, and every
 * launch with it returns RADON_ERR_INVALID_ARG.
 */
typedef struct {
    int n;                   /* image side N */
    const double* angles;    /* host, n_angles radians */
    int n_angles;
    int is_fan;              /* 0 parallel (Section 3.1.1), 1 fan (Section 3.1.2) */
    double source_distance;  /* fan only */
    double det_distance;     /* fan only; <= 0 selects source_distance */
    int det_count;           /* <= 0 selects N */
    double det_spacing;      /* <= 0 selects the default of the geometry kind */
    double step;             /* <= 0 selects 1.0 */
    int host_only;
} radon_geometry_desc;

RADON_API radon_status radon_geometry_create(const radon_geometry_desc* desc, radon_geometry** out);

/*
 * Copies the ray table the kernels read.  For ray r = v * det_count + d, rays[8r..8r+7] =
 * (J0, I0, fx0, fy0, dxh, dyh, dxl, dyl) and counts[r] = number of samples; sample
 * k' = 0..counts[r]-1 sits at x = J0 + fx0 + k' (dxh + dxl), y = I0 + fy0 + k' (dyh + dyl) in
 * pixel-index coordinates (x = column, y = row).  J0, I0 are integers (stored exactly as floats),
 * fx0, fy0 lie in [0, 1) and k' * dxh is exact in FP32 (split precision, so kernels can re-base
 * positions without FP32 drift).  Either pointer may be NULL.  Host buffers of
 * n_angles * det_count entries (x8 floats for rays).
 */
RADON_API radon_status radon_geometry_copy_rays(const radon_geometry* geometry, float* rays, int32_t* counts);

/* Frees the geometry and its device tables (synchronises the device).  NULL is ignored. */
RADON_API void radon_geometry_destroy(radon_geometry* geometry);

typedef struct {
    int n;                   /* image side */
    int n_angles;            /* views */
    int det_count;           /* detector bins */
    int is_fan;              /* 0 parallel, 1 fan */
    double det_spacing;      /* after defaults */
    double step;             /* after defaults */
    double source_distance;  /* 0 for parallel */
    double det_distance;     /* 0 for parallel; after defaults for fan */
    int64_t sample_count;    /* bilinear samples of one image (all rays), FP64 enumeration */
    int device;              /* CUDA device the tables live on */
} radon_geometry_info;

RADON_API radon_status radon_geometry_get_info(const radon_geometry* geometry, radon_geometry_info* out);

/* Number of bilinear samples the forward projection of ONE image evaluates (the throughput
 * unit; the adjoint applies the same weights).  -1 for an invalid handle. */
RADON_API int64_t radon_geometry_sample_count(const radon_geometry* geometry);

/*
 * Forward projection y = A x (Section 3.1.1 / 3.1.2 "forward").
 *   img    device, [batch][N][N] of dtype
 *   sino   device, [batch][n_angles][det_count] of dtype, overwritten
 *   batch  >= 0 (0 is a no-op)
 * Runs the tuned kernels on `stream`; no allocation, no synchronisation.
 */
RADON_API radon_status radon_forward(const radon_geometry* geometry, const void* img, void* sino, radon_dtype dtype,
                           int batch, void* stream);

/*
 * Exact adjoint x = A^T y (Section 3.1.1 / 3.1.2 "backprojection" read as the transpose of
 * the forward; it is also the gradient of the forward, Section 2).
 *   sino   device, [batch][n_angles][det_count] of dtype
 *   img    device, [batch][N][N] of dtype, overwritten
 */
RADON_API radon_status radon_backward(const radon_geometry* geometry, const void* sino, void* img, radon_dtype dtype,
                            int batch, void* stream);

/*
 * Explicit kernel selection (comparison forms and the autotuner).
 *
 * Under RADON_ALGO_AUTO a batch of ONE image with no tile parameters (views_per_cta, rows_per_slab,
 * images_per_cta, tile and threads all 0) runs the single-image kernels -- the uneven-batch plan's
 * per-image forward (one texel load per sample, FP32 weights; it needs the workspace of
 * radon_forward_ws) and adjoint (one weight per candidate ray) -- because a batch-interleaved group
 * would carry the image in one of its 4 to 16 slots: 2-2.6x faster forward and 1.25-1.4x faster
 * adjoint at 512^2.  Larger batches, or explicit parameters, run the batch-interleaved kernels.
 *
 * `weights` selects the forward projection's bilinear-weight precision for FP16 storage (Section
 * 3.3's half-precision path stores in FP16 and computes in single precision):
 *   RADON_WEIGHTS_DEFAULT (0) and RADON_WEIGHTS_F32 (1): FP32 weights, texel values converted to
 *     FP32, FP32 FMAs -- the paper's all-single-precision arithmetic, used by every storage type;
 *   RADON_WEIGHTS_F16 (2, opt-in, FP16 storage only): each sample's four weights are rounded to FP16
 *     and every product of a weight and a texel value is formed exactly in one mixed-precision FMA
 *     accumulated in FP32.  Nothing converts the texel values, so the inner loop runs at the
 *     shared-memory load pipe's rate; the weight rounding (relative <= 2^-12 per weight) shifts a ray
 *     sum by at most 2^-12 of its size, below FP16's own output rounding.  BF16 and FP32 storage, and
 *     every fused call whose epilogue has an addend, keep FP32 weights whatever this field says.
 * Any other value is RADON_ERR_INVALID_ARG.
 */
enum { RADON_WEIGHTS_DEFAULT = 0, RADON_WEIGHTS_F32 = 1, RADON_WEIGHTS_F16 = 2 };

typedef struct {
    int algo;            /* radon_algo */
    int views_per_cta;   /* TILED forward: views per CTA (0 = default: 8, 4, 2, 1 tried in turn, then with two
                            threads per ray where no one-thread shape fits; a fixed value keeps one) */
    int rows_per_slab;   /* TILED forward: image rows staged per step (0 = default) */
    int images_per_cta;  /* TILED: images sharing the geometry work in one CTA (0 = default; the packed
                            adjoint takes 8, 16 or 32, the staged one 4, 8 or 16; the packed forward one
                            or two texel groups: 8 or 16 for 16-bit storage, 4 or 8 for FP32, other
                            values leaving it at its default) */
    int tile;            /* TILED backward: pixel tile side (0 = default) */
    int threads;         /* threads per CTA (0 = default) */
    int weights;         /* forward, FP16 storage: RADON_WEIGHTS_* (0 = default = FP32 weights) */
} radon_launch_config;

RADON_API radon_status radon_forward_ex(const radon_geometry* geometry, const void* img, void* sino, radon_dtype dtype,
                              int batch, const radon_launch_config* config, void* stream);
RADON_API radon_status radon_backward_ex(const radon_geometry* geometry, const void* sino, void* img, radon_dtype dtype,
                               int batch, const radon_launch_config* config, void* stream);

/*
 * Device workspace, in bytes, that radon_forward_ws uses for `batch` images of `dtype`: the batch
 * packed into 16-byte texels holding 4 (FP32) or 8 (16-bit) images each, once in row order and once
 * transposed; for batch 1, at least the single-image forward's quad texels (each pixel's 2 x 2
 * neighbourhood, 16 bytes for FP32 and 8 for 16-bit storage, (N + 1)^2 of them in each of the two
 * frames).  Returns 0 for an invalid geometry, dtype or batch.
 */
RADON_API size_t radon_forward_workspace_size(const radon_geometry* geometry, radon_dtype dtype, int batch);

/*
 * Images per CTA of the packed forward that radon_forward_ws (with a large enough workspace) runs for
 * this call: one texel group (8 for 16-bit storage, 4 for FP32) or two groups whose images share each
 * sample's position, floor and weight evaluation (16 / 8).  By default 16-bit batches of more than 8
 * images take two groups and FP32 one; `config`'s images_per_cta chooses where it holds one of those
 * values.  Where no shape with one thread per ray fits a TMA box (sparse views with a detector wider
 * than the image) and `config` fixes no views per CTA, two threads share each ray (half the detectors
 * per CTA, one texel group).  *images = 0 when another kernel serves the call (one image under AUTO,
 * the PLAIN algorithm, a geometry no packed shape takes).  Host only (host-only geometries are
 * answered too); no launch.
 */
RADON_API radon_status radon_forward_images_per_cta(const radon_geometry* geometry, radon_dtype dtype, int batch,
                                                    const radon_launch_config* config, int* images);

/*
 * Forward projection with a caller-owned device workspace (>= radon_forward_workspace_size bytes,
 * 16-byte aligned, used in stream order on `stream`, contents overwritten).  The batch is packed
 * once into the workspace, then every CTA copies its bands of texels straight into shared memory
 * (the fastest path).  A NULL or too small workspace behaves exactly like radon_forward_ex.
 * Allocates nothing; can be captured in a CUDA graph.
 */
RADON_API radon_status radon_forward_ws(const radon_geometry* geometry, const void* img, void* sino,
                                        radon_dtype dtype, int batch, const radon_launch_config* config,
                                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * Device workspace, in bytes, that radon_backward_ws uses for `batch` sinograms of `dtype`: the
 * batch packed into one row per (group, view, detector), laid out [group][view][detector][row], a row
 * holding the group's images in the storage type (bg 16-bit values, or bg FP32 values and four
 * padding words).  Groups of bg = 8 images for batches of at most 8, 16 up to 16; above that 16 for
 * 16-bit storage when the geometry holds an adjoint weight table, else 32 where whole groups of 32
 * cost less than groups of 16 (a 32-image CTA costs ~1.56x a 16-image one) and their staging fits
 * one CTA's shared memory, else 16.  Returns 0 for an invalid geometry, dtype or batch.
 */
RADON_API size_t radon_backward_workspace_size(const radon_geometry* geometry, radon_dtype dtype, int batch);

/*
 * Exact adjoint with a caller-owned device workspace (>= radon_backward_workspace_size bytes,
 * 16-byte aligned, used in stream order, contents overwritten): the sinogram batch is packed once,
 * then every CTA copies the detector windows of its pixel tile straight into shared memory (the
 * fastest path).  A NULL or too small workspace behaves exactly like radon_backward_ex.  Allocates
 * nothing; can be captured in a CUDA graph.
 */
RADON_API radon_status radon_backward_ws(const radon_geometry* geometry, const void* sino, void* img,
                                         radon_dtype dtype, int batch, const radon_launch_config* config,
                                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * Forward projection that allocates nothing (the paper has no counterpart: this serves callers that
 * cannot allocate device memory -- real-time loops that forbid allocation after start-up, code that
 * must not let an allocation synchronise the device, plain C hosts without a device allocator).  It
 * runs the packed path of radon_forward_ws with its scratch in a fixed 32 MiB device array inside
 * the library instead of a caller workspace.
 *   - Same arguments and results as radon_forward_ws with a workspace.  The limit is the packed
 *     batch, 2 * ceil(batch / BG) * N^2 * 16 bytes (BG = 4 images for FP32 storage, 8 for 16-bit; a
 *     batch of one is one group): a batch that needs more than 32 MiB is rejected with
 *     RADON_ERR_INVALID_ARG -- split it.
 *   - Every GPU that loads the library holds the 32 MiB until the process exits.
 *   - All calls share the array: each call overwrites what the previous one left there (nothing in
 *     it needs to start at zero), and calls whose kernels overlap on the GPU (e.g. on two streams)
 *     race on it -- order them.
 *   - The first call on each device looks up the array's address with that device current and keeps
 *     it for the life of the process; make that first call before any stream capture begins.  The
 *     kept address does not survive a reset of the device's primary context (cudaDeviceReset).
 */
RADON_API radon_status radon_forward_static_scratch(const radon_geometry* geometry, const void* img, void* sino,
                                                    radon_dtype dtype, int batch, void* stream);

/*
 * Weight table of the exact adjoint (a GB300 memory-for-compute trade; the paper computes every weight
 * on the fly).  radon_geometry_build_adjoint_table precomputes, for every 16 x 16 pixel tile, view and
 * vertical pixel pair, the first detector whose ray weighs on the pair and both pixels' bilinear weights
 * on five consecutive rays from it -- the weights the packed adjoint (radon_backward_ws and the calls
 * built on it) would compute, by the same arithmetic.  Pairs whose weighted rays span more than five
 * detectors in a view (rays denser than a pixel, e.g. near a fan's source) are marked and keep
 * computing their weights.  While a geometry holds its table, the packed adjoint of batches that run
 * 8- or 16-image groups reads the weights instead of evaluating them: the same nonzero products added
 * in the same order, so the same bits.
 *   - radon_geometry_adjoint_table_size: the table's device bytes, tiles x views x (128 pairs x 44
 *     + 4) (4.2 GB for 512^2 and 720 views); no allocation.
 *   - radon_geometry_build_adjoint_table: allocates the table on the geometry's device (which must be
 *     current) and fills it; synchronises the device; not capturable.  RADON_ERR_UNSUPPORTED (nothing
 *     kept) where the packed adjoint cannot serve the geometry (a detector window wider than 256 or a
 *     sampling step of sqrt(2) / 3 or less), RADON_ERR_OOM when the device memory runs out.  Building
 *     again replaces the table.
 *   - radon_geometry_adjoint_table_overflow: the fraction of (pair, view) records left to the
 *     on-the-fly weights (0 without a table).
 *   - radon_geometry_free_adjoint_table: frees it (radon_geometry_destroy does too); the adjoint then
 *     computes its weights again.  Calls that may still read the table must have completed.
 */
RADON_API radon_status radon_geometry_adjoint_table_size(const radon_geometry* geometry, size_t* bytes);
RADON_API radon_status radon_geometry_build_adjoint_table(radon_geometry* geometry);
RADON_API radon_status radon_geometry_adjoint_table_overflow(const radon_geometry* geometry, double* fraction);
RADON_API radon_status radon_geometry_free_adjoint_table(radon_geometry* geometry);

/*
 * ---- Iterative reconstruction (Section 4.2: Landweber iteration, step size by power iteration) ----
 *
 * Output epilogue of the fused projections below.  Each output element is
 *     out[i] = op_scale * s * P[i] + add_scale * add[i]
 * where P is the projection (forward or adjoint, as radon_forward / radon_backward compute it),
 * s = *op_scale_dev if op_scale_dev is not NULL (a device FP32 scalar, read by the kernels, so a
 * step length can stay on the device) and 1 otherwise, and `add` is an optional device array of the
 * output's dtype and layout (NULL: no addend).  `add` may be the output buffer itself (in-place
 * update); otherwise it must not overlap the output.  The sum is formed in FP32 and rounded once to
 * the storage type, so a 16-bit residual A x - y keeps its own relative precision instead of
 * inheriting the rounding of A x.  {1, NULL, 0, NULL} gives exactly radon_forward / radon_backward.
 * Landweber's update x - alpha A^T (A x - y) is two calls:
 *     r  = forward_fused(x,  {1, NULL, -1, y})
 *     x' = backward_fused(r, {-1, alpha_dev, 1, x}).
 */
typedef struct radon_epilogue {
    float op_scale;
    const float* op_scale_dev;
    float add_scale;
    const void* add;
} radon_epilogue;

/*
 * Forward projection / exact adjoint with an output epilogue (NULL `epilogue` = identity).
 * Otherwise the same as radon_forward_ws / radon_backward_ws: optional launch config, optional
 * caller workspace (NULL or too small: the paths that need none).  `add` must be aligned to its
 * element size and `op_scale_dev` to 4 bytes.  Allocates nothing; can be captured.
 */
RADON_API radon_status radon_forward_fused(const radon_geometry* geometry, const void* img, void* sino,
                                           radon_dtype dtype, int batch, const radon_epilogue* epilogue,
                                           const radon_launch_config* config, void* workspace,
                                           size_t workspace_bytes, void* stream);
RADON_API radon_status radon_backward_fused(const radon_geometry* geometry, const void* sino, void* img,
                                            radon_dtype dtype, int batch, const radon_epilogue* epilogue,
                                            const radon_launch_config* config, void* workspace,
                                            size_t workspace_bytes, void* stream);

/* Device workspace, in bytes, of radon_dot. */
RADON_API size_t radon_dot_workspace_size(void);

/*
 * Inner product of two device arrays of `count` elements of `dtype` (the same for both):
 *     *result = scale * <a, b> + (accumulate ? *result : 0)
 * with `result` one device FP32.  Products are summed in FP32 per thread and in FP64 across
 * threads and blocks, in a fixed order: the result is deterministic.  Two kernels, in stream order,
 * using the caller's workspace (>= radon_dot_workspace_size bytes, 8-byte aligned).  Allocates
 * nothing; can be captured.
 */
RADON_API radon_status radon_dot(const void* a, const void* b, radon_dtype dtype, int64_t count, float scale,
                                 float* result, int accumulate, void* workspace, size_t workspace_bytes,
                                 void* stream);

/*
 * y = alpha * s * x + beta * y over `count` elements, elementwise, with x of dtype `x_dtype` and y of
 * `y_dtype` (they may differ: this also casts), s = *alpha_dev if alpha_dev is not NULL, else 1.
 * With beta == 0, y is written without being read (it may hold anything, NaN included).  FP32
 * arithmetic, one rounding to y's type.  Allocates nothing; can be captured.
 */
RADON_API radon_status radon_axpby(const void* x, radon_dtype x_dtype, void* y, radon_dtype y_dtype, int64_t count,
                                   float alpha, const float* alpha_dev, float beta, void* stream);

/*
 * Device workspace, in bytes, of radon_power_iteration for this geometry (FP32 image and
 * sinogram buffers, the projections' packed workspaces and the dot workspace).
 */
RADON_API size_t radon_power_iteration_workspace_size(const radon_geometry* geometry);

/*
 * Largest eigenvalue of A^T A by the power method, the step-size estimate of Landweber's iteration:
 *     z = v0 / |v0|;  repeat `iterations` times:  w = A^T A z,  lambda = <z, w>,  z = w / |w|
 * (lambda is the Rayleigh quotient of the last iterate).  v0 is one FP32 image [N][N] on the device
 * (the caller draws it, e.g. N(0, 1) from a seeded generator; it is not modified).  All arithmetic
 * runs in FP32 storage on the device; *lambda_out (one device FP32) receives the estimate and, if
 * alpha_out is not NULL, *alpha_out receives Landweber's step alpha = 1 / lambda.  Workspace:
 * >= radon_power_iteration_workspace_size bytes, 16-byte aligned.  Allocates nothing, never
 * synchronises; can be captured.  A zero v0 or an operator that maps z to zero gives NaN.
 */
RADON_API radon_status radon_power_iteration(const radon_geometry* geometry, const float* v0, int iterations,
                                             float* lambda_out, float* alpha_out, void* workspace,
                                             size_t workspace_bytes, void* stream);

/*
 * Synchronises `stream`, then reads and clears the library's device error word.
 * Returns RADON_OK, RADON_ERR_TIMEOUT or RADON_ERR_DEVICE_BOUNDS (from kernels), or
 * RADON_ERR_CUDA if the synchronisation itself failed.
 */
RADON_API radon_status radon_get_device_error(void* stream);

/*
 * Pixel-driven interpolating backprojector (the kind of backprojection the paper's comparisons use,
 * Section 3.1): img[b][i][j] = sum_v |grad t_v| * sino[b][v] linearly interpolated at t_v(j, i), where
 * t_v is the continuous detector index of the pixel centre (parallel: (c . n) / ds + (D-1)/2; fan:
 * where the source-to-pixel line meets the flat detector) and |grad t_v| the density of rays there in
 * bins per pixel (1 / ds for parallel beams); bins outside [0, D) read as zero.  It approximates the
 * exact adjoint (radon_backward) at a fraction of the cost but is not its transpose.  Same buffers and
 * rules as radon_backward; allocates nothing; can be captured.
 */
RADON_API radon_status radon_backproject_interpolating(const radon_geometry* geometry, const void* sino, void* img,
                                                       radon_dtype dtype, int batch, void* stream);

/*
 * The same with a caller workspace (>= radon_backward_workspace_size bytes, 16-byte aligned): the
 * sinogram batch is packed once and every 16 x 16 tile's detector windows arrive in shared memory by
 * TMA through the exact adjoint's pipeline, two interpolation taps per pixel and view.  A NULL or too
 * small workspace, or a shape that pipeline refuses, falls back to radon_backproject_interpolating.
 */
RADON_API radon_status radon_backproject_interpolating_ws(const radon_geometry* geometry, const void* sino, void* img,
                                                          radon_dtype dtype, int batch, void* workspace,
                                                          size_t workspace_bytes, void* stream);

/*
 * ---- Conjugate-gradient solvers (Section 2.1's solvers module, Section 4.2; M. Hanke, "Conjugate
 * gradient type methods for ill-posed problems") ----
 *
 * Batched vector kernels with one scalar per item, for per-image conjugate-gradient recursions:
 *   radon_dot_batched:   result[i] = scale <a_i, b_i> (+ result[i] if accumulate), items of `count`
 *                        elements, deterministic (FP32 per thread, FP64 across threads and blocks);
 *                        workspace >= radon_dot_batched_workspace_size(batch) bytes, 8-byte aligned;
 *   radon_axpby_batched: y_i = alpha s_i x_i + beta t_i y_i, s_i = alpha_dev[i] (NULL: 1),
 *                        t_i = beta_dev[i] (NULL: 1); y is not read when beta == 0 and beta_dev NULL;
 *   radon_safe_divide:   out[i] = num[i] / den[i] where den[i] > 0, else 0 (device FP32 arrays).
 * All allocate nothing and can be captured; batch <= 65535 for the dot.
 */
RADON_API size_t radon_dot_batched_workspace_size(int batch);
RADON_API radon_status radon_dot_batched(const void* a, const void* b, radon_dtype dtype, int batch, int64_t count,
                                         float scale, float* result, int accumulate, void* workspace,
                                         size_t workspace_bytes, void* stream);
RADON_API radon_status radon_axpby_batched(const void* x, radon_dtype x_dtype, void* y, radon_dtype y_dtype,
                                           int batch, int64_t count, float alpha, const float* alpha_dev, float beta,
                                           const float* beta_dev, void* stream);
RADON_API radon_status radon_safe_divide(const float* num, const float* den, float* out, int batch, void* stream);

/*
 * CGNE: conjugate gradients on the normal equation A^T A x = A^T y, every image its own problem:
 *   r = y - A x;  s = A^T r;  p = s;  gamma = |s|^2;  per iteration:
 *   q = A p;  alpha = gamma / |q|^2;  x += alpha p;  r -= alpha q;  s = A^T r;
 *   gamma' = |s|^2;  p = s + (gamma' / gamma) p;  gamma = gamma'
 * (a zero denominator gives a zero step).  x ([batch][N][N], FP32) holds the start on entry and the
 * iterate after `iterations` steps on return; y is the FP32 sinogram batch.  Runs entirely on the
 * device in stream order with the caller's workspace (>= radon_cgne_workspace_size bytes, 16-byte
 * aligned): allocates nothing, never synchronises, can be captured.  FP32 storage only
 * (RADON_ERR_UNSUPPORTED otherwise): the recursion's orthogonality does not survive 16-bit vectors.
 */
RADON_API size_t radon_cgne_workspace_size(const radon_geometry* geometry, int batch);
RADON_API radon_status radon_cgne(const radon_geometry* geometry, const void* y, void* x, radon_dtype dtype, int batch,
                                  int iterations, void* workspace, size_t workspace_bytes, void* stream);

/*
 * ---- Filtered backprojection (Section 3.1.3) ----
 *
 * Each view's projection is filtered along the detector in the frequency domain by the DFT of the
 * band-limited ramp kernel of Kak & Slaney (Chapter 3, Eq. 61: 1/4 at offset 0, -1/(pi^2 m^2) at odd
 * offsets m, 0 at even ones) zero-padded to P = the smallest power of two >= max(2D - 1, 2), times a window
 * of the normalised frequency f in [-1/2, 1/2] cycles per bin, and scaled by pi / V; the exact
 * adjoint of the result is the reconstruction (parallel beam; no fan-beam weighting is applied).
 */
typedef enum {
    RADON_FILTER_RAM_LAK = 0,   /* window 1 */
    RADON_FILTER_SHEPP_LOGAN,   /* sin(pi f) / (pi f) */
    RADON_FILTER_COSINE,        /* cos(pi f) */
    RADON_FILTER_HAMMING,       /* 0.54 + 0.46 cos(2 pi f) */
    RADON_FILTER_HANN           /* 0.5 + 0.5 cos(2 pi f) */
} radon_filter;

/*
 * out = the filtered sinogram batch ([batch][V][D], same dtype as `sino`, FP32 arithmetic).  The
 * zero-padded circular convolution equals a linear one over the D bins, so the kernel sums it
 * directly with taps precomputed in FP64 when the geometry was created (the two routes agree to
 * rounding).  `out` must not overlap `sino`.  Allocates nothing; can be captured.
 */
RADON_API radon_status radon_filter_sinogram(const radon_geometry* geometry, const void* sino, void* out,
                                             radon_dtype dtype, int batch, radon_filter filter, void* stream);

/*
 * ---- Uneven batches in one persistent launch (Section 4.1: batch processing, here of images of
 * different sizes, each with its own geometry) ----
 *
 * A plan covers n items; item i projects (direction 0) or back-projects (direction 1) items[i].batch
 * images with geometry items[i].geometry from items[i].in to items[i].out (device buffers laid out as
 * for radon_forward / radon_backward).  Every image of every item becomes a unit; the plan splits the
 * units into work items -- blocks of rays (forward) or 16 x 16 pixel tiles (adjoint) -- ordered
 * largest first, and one persistent kernel (one CTA per SM slot) takes them from a device counter
 * until the list is empty, so small and large images share the GPU without a tail of idle SMs.
 *   - Forward: the plan keeps a packed copy of every image (each pixel's 2 x 2 bilinear neighbourhood
 *     in one 8-byte texel, FP32: 16 bytes, in the image frame and transposed), refreshed by a pack
 *     kernel at every launch; each sample is one texel load.
 *   - Adjoint: per chunk of views the CTA stages the sinogram values of the rays crossing its tile in
 *     shared memory (re-basing one ray per parallel-beam view, whose rays share one sample lattice,
 *     or every ray of a fan-beam window), then every thread gathers its pixel.
 *   - Tile shapes (forward: views per ray block x lanes per ray, 8 candidates; adjoint: views per
 *     chunk, 4 candidates) are picked per image size and geometry kind by a built-in autotuner that
 *     times each candidate on the plan's own buffers at creation (and writes the outputs while doing
 *     so), unless options fix them.  With the environment variable RADON_TUNE_CACHE naming a file,
 *     picks are appended to it and later plans reuse them for the same direction, storage type, image
 *     size and geometry kind instead of timing.
 * The caller keeps the geometries and buffers alive until radon_batch_plan_destroy; the buffer
 * addresses are baked into the plan.
 */
typedef struct radon_item {
    const radon_geometry* geometry;
    const void* in;
    void* out;
    int batch;
} radon_item;

typedef struct radon_plan radon_plan;

typedef struct radon_plan_options {
    int autotune;            /* 1: time the candidates (default); 0: library defaults */
    int forward_views;       /* > 0: views per forward ray block (1, 2, 4 or 8; detectors = 256 / (views x lanes)) */
    int adjoint_views;       /* > 0: views per adjoint chunk (4, 8, 16 or 32; RADON_ERR_UNSUPPORTED if 32
                                views of the widest detector window do not fit one CTA's shared memory) */
    int forward_lanes;       /* > 0: lanes per forward ray (1, or 4: the ray's samples interleaved over four
                                lanes whose partial sums meet in a fixed shuffle tree) */
    int forward_rows;        /* > 0: texel rows per slab of the staged forward (8, 16 or 32) */
    int forward_kernel;      /* 0: the staged forward (image slabs copied into shared memory by bulk copies)
                                where its bands fit, else the L1 gather; 1: staged (RADON_ERR_UNSUPPORTED if
                                the bands do not fit); -1: the L1 gather (one texel load per sample) */
} radon_plan_options;

/*
 * Builds a plan (allocates device memory, uploads the work list, autotunes; synchronises; not
 * capturable).  All items share `dtype` and must live on the current device; items with batch 0 are
 * skipped.  `options` may be NULL (autotune on).  RADON_ERR_INVALID_ARG for a bad item (NULL or
 * host-only geometry, NULL buffer, batch < 0), RADON_ERR_OOM if device memory runs out.
 */
RADON_API radon_status radon_batch_plan_create(const radon_item* items, int n, int direction, radon_dtype dtype,
                                               const radon_plan_options* options, radon_plan** out);

/*
 * Runs the plan on `stream`: resets the work counter, packs (forward), then one persistent kernel.
 * Allocates nothing, never synchronises; can be captured in a CUDA graph (replays read the items'
 * input buffers as they are at replay time).  A plan owns one work counter and (forward) one packed
 * texel buffer, so launches of the same plan must be ordered on the GPU (one stream, or events
 * between streams; graph replays of it likewise); concurrent use needs one plan per launch.
 */
RADON_API radon_status radon_batch_plan_launch(radon_plan* plan, void* stream);

/* What the plan built: units (images), work items, persistent CTAs, and the tile shape of item i. */
typedef struct radon_plan_info {
    int units;
    int work_items;
    int ctas;
    int direction;
} radon_plan_info;
RADON_API radon_status radon_batch_plan_get_info(const radon_plan* plan, radon_plan_info* info);
RADON_API radon_status radon_batch_plan_item_config(const radon_plan* plan, int item, int* views);
/* The shape item i runs with: views per forward ray block or adjoint chunk, and lanes per forward ray
 * (1 for the adjoint). */
RADON_API radon_status radon_batch_plan_item_shape(const radon_plan* plan, int item, int* views, int* lanes);

/* Texel rows per slab of item i's staged forward (0 for the L1 gather and for adjoint plans). */
RADON_API radon_status radon_batch_plan_item_rows(const radon_plan* plan, int item, int* rows);

RADON_API void radon_batch_plan_destroy(radon_plan* plan);

/*
 * Measures the achievable rate of the forward projection's inner loop on the current GPU: a kernel
 * that marches straight rays through a shared-memory-resident tile of batch-interleaved texels (four
 * 16-byte loads per texel group, one floor / weight evaluation and FP32 accumulation for every image
 * of the texels per sample, no geometry, no TMA) on every SM, with the forward's own accumulation
 * code for `dtype` storage and the `weights` setting of radon_launch_config (RADON_WEIGHTS_F16 for
 * FP16 storage only), over `groups` (1 or 2) texel groups per sample as the packed forward's CTAs
 * take them (radon_forward_images_per_cta).  *samples_per_second receives image-samples per second
 * (one probe sample serves the 8 (16-bit) or 4 (F32) images of each texel group), the ceiling the
 * forward's measured rate is compared with.  Synchronises the device; not capturable.
 * radon_probe_gather_ceiling_ex(dtype, weights, out) takes one group;
 * radon_probe_gather_ceiling(dtype, out) is radon_probe_gather_ceiling_ex(dtype, RADON_WEIGHTS_DEFAULT, out).
 */
RADON_API radon_status radon_probe_gather_ceiling_groups(radon_dtype dtype, int weights, int groups,
                                                         double* samples_per_second);
RADON_API radon_status radon_probe_gather_ceiling_ex(radon_dtype dtype, int weights, double* samples_per_second);
RADON_API radon_status radon_probe_gather_ceiling(radon_dtype dtype, double* samples_per_second);

/*
 * Number of kernels this library has launched in this process so far (every pack, projection and
 * vector kernel, counted on the host when the launch is issued).  Thread-safe; for accounting, e.g.
 * the launches inside a timed region are the difference of two reads.
 */
RADON_API uint64_t radon_kernel_launch_count(void);

/* Static, never NULL. */
RADON_API const char* radon_status_string(radon_status status);

/* Thread-local text of the last failure on this thread ("" if none).  Valid until the next call. */
RADON_API const char* radon_last_error_message(void);

/* RADON_ABI_VERSION of the loaded library. */
RADON_API int radon_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RADON_H */
