// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "radon.h"

namespace radon {

constexpr uint64_t kGeometryMagic = 0x5241444f4e47454fULL;  // "RADONGEO"

// Exactness margin of the split ray table, in pixels beyond either end of a ray.
constexpr int kSplitMarginPx = 24;

// One ray in pixel-index coordinates (column x = j, row y = i), stored in split precision so
// kernels can re-base sample positions without FP32 drift.  Sample k' = 0..nk-1 sits at
//     x = J0 + fx0 + k' (dxh + dxl),   y = I0 + fy0 + k' (dyh + dyl)
// with J0, I0 integers, fx0, fy0 in [0, 1), and the step split so that k' * dxh is exact in
// FP32 for every k' in [-M, nk + M) (dxh carries at most 24 - ceil(log2(nk + M)) significant
// bits, M = kSplitMarginPx / h + 8 samples) while dxl holds the remainder.  The ray is oriented
// so that its major-axis step is >= 0: the y step for views of the vertical class, the x step
// for the horizontal class.
struct RayT {
    int J0, I0;
    float fx0, fy0;
    float dxh, dyh, dxl, dyl;
};

// Per-view projective map from a point (x = j, y = i, index coordinates) to the continuous
// detector index t: t = (ax*x + ay*y + a0) / (bx*x + by*y + b0).  Ray d crosses t = d.
struct ViewF {
    float ax, ay, a0, bx, by, b0;
    int major;   // 0: |u_y| >= |u_x| (rays run mostly along rows' normal, "vertical"); 1: horizontal
    int pad;
};

// Output epilogue applied by every projector kernel at its store:
//     out[i] = op_scale * s * P[i] + add_scale * add[i]
// with P the projection (already multiplied by the step h), s = *op_scale_dev when that pointer
// is set (a device scalar, e.g. a step length that stays on the device), and add an optional
// addend in the output's dtype and layout (it may be the output buffer itself).  The identity
// {1, NULL, 0, NULL} leaves P unchanged bit for bit.
struct Epilogue {
    float op_scale;
    const float* op_scale_dev;
    float add_scale;
    const void* add;
};

inline Epilogue identity_epilogue() { return Epilogue{1.0f, nullptr, 0.0f, nullptr}; }

struct Int2 {
    int x, y;
};

}  // namespace radon

struct radon_geometry {
    uint64_t magic = 0;
    int n = 0, V = 0, D = 0, fan = 0, device = -1, host_only = 0;
    double ds = 1.0, h = 1.0, S = 0.0, Ddet = 0.0;
    int64_t samples = 0;
    int max_nk = 0;
    int bwd_window = 0;               // widest detector window of a 16x16 tile (tiled adjoint)
    int fwd_pair_views = 0;           // tiled forward: two views x four detectors per load phase
    std::vector<radon::Int2> h_groups;  // view groups for G = 1, 2, 4, 8 (concatenated)
    int group_offset[4] = {0, 0, 0, 0};
    int group_count[4] = {0, 0, 0, 0};
    radon::Int2* d_groups = nullptr;
    // widest working band of the tiled forward per (views/CTA, detectors/CTA, rows/slab)
    std::mutex band_mu;
    std::map<long long, int> band_width;
    std::vector<double> angles;
    std::vector<radon::RayT> h_ray;   // [V*D]
    std::vector<int> h_nk;            // [V*D]
    std::vector<radon::ViewF> h_view; // [V]
    radon::RayT* d_ray = nullptr;
    int* d_nk = nullptr;
    radon::ViewF* d_view = nullptr;
    // FBP filter taps, (pi / V) k[m] for m = -(D-1) .. D-1 as (hi, lo) FP32 pairs, one row of 2D - 1
    // per radon_filter kind
    float2* d_filter_taps = nullptr;
    // Weight table of the exact adjoint (built on request, radon_geometry_build_adjoint_table):
    // [tile][view][pair] two float4 and one float2 of weights and an int32 first ray; NULL when absent
    void* d_tab_w = nullptr;
    void* d_tab_w5 = nullptr;
    int* d_tab_la = nullptr;
    int* d_tab_vflag = nullptr;   // [tile][view]: some pair of the tile overflows the table there
    int tab_kw = 0;             // samples per candidate window it was built for
    int tab_wd = 0;             // detector window it was built for
    size_t tab_bytes = 0;
    double tab_overflow = 0.0;  // fraction of (pair, view) records left to the on-the-fly weights
};

namespace radon {

// radon_api.cpp: host-side validation and error reporting shared by the entry points
radon_status fail(radon_status st, const std::string& msg);
radon_status cuda_fail(cudaError_t e, const char* what);
radon_status validate_call(const radon_geometry* g, const void* in, const void* out, radon_dtype dt, int batch);
radon_status check_device(const radon_geometry* g);
// The projection dispatcher behind every entry point: packed (with a workspace), tiled, then plain
// kernels, in that order of preference; `epi` NULL = identity epilogue.
radon_status project(const radon_geometry* g, const void* in, void* out, radon_dtype dt, int batch,
                     const radon_launch_config* cfg, void* stream, bool forward, void* ws, size_t ws_bytes,
                     const radon_epilogue* epi);

// geometry.cpp
radon_status build_geometry(radon_geometry* g);  // fills host tables and sample count
int backward_window_width(const radon_geometry* g, int tile);
// widest band (compute-frame columns, before alignment) of the tiled forward; cached per config
int forward_band_width(radon_geometry* g, int G, int Dt, int R);
const char* set_error(const std::string& msg);   // thread-local message, returns it

// kernels_plain.cu
cudaError_t launch_forward_plain(const radon_geometry* g, const void* img, void* sino, radon_dtype dt, int batch,
                                 int threads, const Epilogue& ep, cudaStream_t s);
cudaError_t launch_backward_plain(const radon_geometry* g, const void* sino, void* img, radon_dtype dt, int batch,
                                  int threads, const Epilogue& ep, cudaStream_t s);

// backward_tiled.cu: RADON_ERR_UNSUPPORTED if the geometry / buffers do not fit the tiled kernel
radon_status launch_backward_tiled(const radon_geometry* g, const void* sino, void* img, radon_dtype dt, int batch,
                                   int images_per_cta, const Epilogue& ep, cudaStream_t s, std::string* why);

// forward_tiled.cu: RADON_ERR_UNSUPPORTED if the geometry / buffers do not fit the tiled kernel
radon_status launch_forward_tiled(radon_geometry* g, const void* img, void* sino, radon_dtype dt, int batch,
                                  const radon_launch_config* cfg, const Epilogue& ep, cudaStream_t s,
                                  std::string* why);

// forward_tiled.cu: the packed forward's launch shape for a call (views per CTA from cfg or 8, image
// groups per CTA, rows per slab, band width, ring stages, shared memory) with `lanes` (1 or 2) threads
// per ray; RADON_ERR_UNSUPPORTED with the reason if the geometry does not fit it.  `fp16_weights`: the
// FP16-weight mode will run.  Two lanes per ray halve the detectors of a CTA (narrower bands, for views
// too sparse or detectors too wide for one lane) and take one texel group.
struct PackedFwdShape {
    int G, Dt, NG, LN, R, wbox, stages;
    size_t smem;
};
radon_status packed_forward_shape(radon_geometry* g, radon_dtype dt, int batch, const radon_launch_config* cfg,
                                  bool fp16_weights, int lanes, PackedFwdShape* out, std::string* why);

// forward_tiled.cu: the packed-input forward (the workspace already holds pack_images' output)
radon_status launch_forward_packed(radon_geometry* g, const void* packed, void* sino, radon_dtype dt, int batch,
                                   const radon_launch_config* cfg, const Epilogue& ep, cudaStream_t s,
                                   std::string* why, int lanes = 1);

// batch_plan.cu: one image (a batch-1 call) through the uneven-batch plan's kernels -- one texel load
// per forward sample, one weight per adjoint candidate -- instead of a batch-interleaved group that
// the image would fill to one eighth.  The forward packs the image's quad texels into `ws`
// (single_forward_workspace_bytes, 16-byte aligned); the adjoint needs no workspace.
size_t single_forward_workspace_bytes(const radon_geometry* g, radon_dtype dt);
radon_status launch_forward_single(const radon_geometry* g, const void* img, void* sino, radon_dtype dt, void* ws,
                                   const Epilogue& ep, cudaStream_t s);
radon_status launch_backward_single(const radon_geometry* g, const void* sino, void* img, radon_dtype dt,
                                    const Epilogue& ep, cudaStream_t s, std::string* why);

// pack.cu
size_t packed_image_bytes(int n, int batch, radon_dtype dt);
cudaError_t launch_pack_images(const void* img, void* workspace, int n, int batch, radon_dtype dt, cudaStream_t s);
size_t packed_sino_bytes(int V, int D, int batch, int bg, radon_dtype dt);
cudaError_t launch_pack_sino(const void* sino, void* workspace, int V, int D, int batch, int bg, radon_dtype dt,
                             cudaStream_t s);

// backward_packed.cu: the packed-sinogram adjoint (the workspace already holds pack_sino's output)
int backward_packed_images_per_cta(const radon_geometry* g, int batch, radon_dtype dt, const radon_launch_config* cfg);
// backward_packed.cu: the exact adjoint's weight table of a geometry (bytes it needs; build; free)
size_t adjoint_table_bytes(const radon_geometry* g);
radon_status build_adjoint_table(radon_geometry* g, std::string* why);
void free_adjoint_table(radon_geometry* g);
radon_status launch_backward_packed(const radon_geometry* g, const void* packed, void* img, radon_dtype dt, int batch,
                                    int images_per_cta, const Epilogue& ep, cudaStream_t s, std::string* why,
                                    bool interpolating = false);

// radon_api.cpp: process-wide count of kernels the library has launched (radon_kernel_launch_count)
void count_launches(int kernels);

// filter.cu: the FBP filter taps of every kind, computed in FP64 and uploaded at geometry creation
radon_status upload_filter_taps(radon_geometry* g);

// kernels_common.cu
cudaError_t read_and_clear_device_error(int* out);
cudaError_t device_error_address(int** out);
int* device_error_word();   // cached per device; NULL on failure

}  // namespace radon
