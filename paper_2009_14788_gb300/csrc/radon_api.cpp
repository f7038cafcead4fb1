// C ABI of libradon (declared in include/radon.h): argument validation, geometry lifetime,
// kernel dispatch and error reporting.  Every argument check runs on the host before any CUDA
// call, so a bad request never reaches the GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "radon_internal.h"

namespace radon {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void count_launches(int kernels) { g_launches.fetch_add((uint64_t)kernels, std::memory_order_relaxed); }

const char* set_error(const std::string& msg) {
    g_last_error = msg;
    return g_last_error.c_str();
}

radon_status fail(radon_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

radon_status cuda_fail(cudaError_t e, const char* what) {
    return fail(RADON_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

bool env_flag(const char* name) {
    const char* v = std::getenv(name);
    return v != nullptr && v[0] != '\0' && std::strcmp(v, "0") != 0;
}

radon_status validate_geometry(const radon_geometry* g) {
    if (g == nullptr) return fail(RADON_ERR_INVALID_ARG, "geometry is NULL");
    if (g->magic != kGeometryMagic) return fail(RADON_ERR_INVALID_ARG, "geometry handle is not a live geometry");
    return RADON_OK;
}

radon_status check_device(const radon_geometry* g) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != g->device)
        return fail(RADON_ERR_INVALID_ARG, "geometry lives on device " + std::to_string(g->device) +
                                               " but device " + std::to_string(dev) + " is current");
    return RADON_OK;
}

radon_status validate_call(const radon_geometry* g, const void* in, const void* out, radon_dtype dt, int batch) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (dt != RADON_F32 && dt != RADON_F16 && dt != RADON_BF16)
        return fail(RADON_ERR_INVALID_ARG, "dtype must be RADON_F32, RADON_F16 or RADON_BF16");
    if (batch < 0) return fail(RADON_ERR_INVALID_ARG, "batch must be >= 0");
    if (batch > 0 && (in == nullptr || out == nullptr)) return fail(RADON_ERR_INVALID_ARG, "NULL buffer with batch > 0");
    if (batch > 0 && in == out) return fail(RADON_ERR_INVALID_ARG, "input and output must not alias");
    const int64_t npix = (int64_t)g->n * g->n, nsino = (int64_t)g->V * g->D;
    if ((int64_t)batch * std::max(npix, nsino) > ((int64_t)1 << 40))
        return fail(RADON_ERR_INVALID_ARG, "batch too large");
    return RADON_OK;
}

radon_status upload(radon_geometry* g) {
    cudaError_t e;
    const size_t nr = g->h_ray.size();
    if ((e = cudaMalloc(&g->d_ray, std::max<size_t>(1, nr) * sizeof(RayT))) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(RADON_ERR_OOM, "device allocation of ray table failed")
                                              : cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&g->d_nk, std::max<size_t>(1, nr) * sizeof(int))) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(RADON_ERR_OOM, "device allocation of count table failed")
                                              : cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&g->d_view, std::max<size_t>(1, g->h_view.size()) * sizeof(ViewF))) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(RADON_ERR_OOM, "device allocation of view table failed")
                                              : cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(g->d_ray, g->h_ray.data(), nr * sizeof(RayT), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy ray table");
    if ((e = cudaMemcpy(g->d_nk, g->h_nk.data(), nr * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy count table");
    if ((e = cudaMemcpy(g->d_view, g->h_view.data(), g->h_view.size() * sizeof(ViewF), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "cudaMemcpy view table");
    if ((e = cudaMalloc(&g->d_groups, std::max<size_t>(1, g->h_groups.size()) * sizeof(Int2))) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(RADON_ERR_OOM, "device allocation of view groups failed")
                                              : cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(g->d_groups, g->h_groups.data(), g->h_groups.size() * sizeof(Int2), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "cudaMemcpy view groups");
    return upload_filter_taps(g);
}

void release(radon_geometry* g) {
    if (g == nullptr) return;
    if (g->d_ray) cudaFree(g->d_ray);
    if (g->d_nk) cudaFree(g->d_nk);
    if (g->d_view) cudaFree(g->d_view);
    if (g->d_groups) cudaFree(g->d_groups);
    if (g->d_filter_taps) cudaFree(g->d_filter_taps);
    free_adjoint_table(g);
    g->magic = 0;
    delete g;
}

radon_status create_common(int n, const double* angles, int n_angles, int det_count, double det_spacing, double step,
                           int fan, double S, double Ddet, int host_only, radon_geometry** out) {
    if (out == nullptr) return fail(RADON_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 8192) return fail(RADON_ERR_INVALID_ARG, "n must be in [1, 8192]");
    if (angles == nullptr) return fail(RADON_ERR_INVALID_ARG, "angles is NULL");
    if (n_angles < 1 || n_angles > (1 << 20)) return fail(RADON_ERR_INVALID_ARG, "n_angles must be in [1, 2^20]");
    for (int v = 0; v < n_angles; ++v)
        if (!std::isfinite(angles[v])) return fail(RADON_ERR_INVALID_ARG, "angles must be finite");
    if (det_count <= 0) det_count = n;
    if (det_count > (1 << 20)) return fail(RADON_ERR_INVALID_ARG, "det_count must be <= 2^20");
    if ((int64_t)det_count * n_angles > ((int64_t)1 << 31))
        return fail(RADON_ERR_INVALID_ARG, "n_angles * det_count must be <= 2^31");
    if (!std::isfinite(step)) return fail(RADON_ERR_INVALID_ARG, "step must be finite");
    if (step <= 0.0) step = 1.0;
    if (step < 1e-3) return fail(RADON_ERR_INVALID_ARG, "step must be >= 1e-3 pixels");
    if (!std::isfinite(det_spacing)) return fail(RADON_ERR_INVALID_ARG, "det_spacing must be finite");
    if (fan) {
        if (!std::isfinite(S) || S <= 0.0) return fail(RADON_ERR_INVALID_ARG, "source_distance must be finite and > 0");
        if (!std::isfinite(Ddet)) return fail(RADON_ERR_INVALID_ARG, "det_distance must be finite");
        if (Ddet <= 0.0) Ddet = S;
        // The source must lie outside the support disk so every ray enters the image once.
        if (S <= 0.5 * (double)(n + 1) * std::sqrt(2.0) + 1.0)
            return fail(RADON_ERR_UNSUPPORTED, "source_distance must exceed (n+1)/sqrt(2) + 1 (source outside the image)");
        if (det_spacing <= 0.0) det_spacing = (S + Ddet) / S * (double)n / (double)det_count;
    } else {
        S = 0.0;
        Ddet = 0.0;
        if (det_spacing <= 0.0) det_spacing = 1.0;
    }
    if (env_flag("RADON_FAULT_INJECT_OOM")) return fail(RADON_ERR_OOM, "allocation failure injected (RADON_FAULT_INJECT_OOM)");

    radon_geometry* g = new (std::nothrow) radon_geometry();
    if (g == nullptr) return fail(RADON_ERR_OOM, "host allocation failed");
    g->n = n;
    g->V = n_angles;
    g->D = det_count;
    g->fan = fan;
    g->ds = det_spacing;
    g->h = step;
    g->S = S;
    g->Ddet = Ddet;
    g->host_only = host_only ? 1 : 0;
    try {
        g->angles.assign(angles, angles + n_angles);
        radon_status st = build_geometry(g);
        if (st != RADON_OK) {
            release(g);
            return st;
        }
    } catch (const std::bad_alloc&) {
        release(g);
        return fail(RADON_ERR_OOM, "host allocation of geometry tables failed");
    }
    if (g->host_only) {
        g->magic = kGeometryMagic;
        *out = g;
        return RADON_OK;
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        release(g);
        return cuda_fail(e, "cudaGetDevice");
    }
    radon_status st = upload(g);
    if (st != RADON_OK) {
        release(g);
        return st;
    }
    g->magic = kGeometryMagic;
    *out = g;
    return RADON_OK;
}

namespace {

radon_status validate_epilogue(const radon_epilogue* e, radon_dtype dt) {
    if (e == nullptr) return RADON_OK;
    const size_t esz = dt == RADON_F32 ? 4 : 2;
    if (e->add != nullptr && ((uintptr_t)e->add % esz) != 0)
        return fail(RADON_ERR_INVALID_ARG, "epilogue addend is not aligned to its element size");
    if (e->op_scale_dev != nullptr && ((uintptr_t)e->op_scale_dev % 4) != 0)
        return fail(RADON_ERR_INVALID_ARG, "epilogue op_scale_dev is not 4-byte aligned");
    if (!std::isfinite(e->op_scale) || !std::isfinite(e->add_scale))
        return fail(RADON_ERR_INVALID_ARG, "epilogue scales must be finite");
    return RADON_OK;
}

}  // namespace

// The packed forward's config for shape candidate i (views per CTA 8, 4, 2, 1 in order unless the caller
// fixed them); images per CTA: one texel group or two (a value meant for the adjoint leaves the default).
radon_launch_config packed_forward_config(const radon_launch_config* cfg, radon_dtype dt, int i) {
    static const int kViewsPacked[4] = {8, 4, 2, 1};
    const bool fixed = cfg != nullptr && cfg->views_per_cta != 0;
    const int bg = dt == RADON_F32 ? 4 : 8;
    const int ipc = cfg != nullptr && (cfg->images_per_cta == bg || cfg->images_per_cta == 2 * bg)
                        ? cfg->images_per_cta : 0;
    return radon_launch_config{RADON_ALGO_TILED, fixed ? cfg->views_per_cta : kViewsPacked[i],
                               cfg ? cfg->rows_per_slab : 0, ipc, 0, 0, cfg ? cfg->weights : 0};
}

// One image under AUTO with no tile parameters runs the single-image kernels.
bool single_image_call(const radon_launch_config* cfg, int batch) {
    const int algo = cfg ? cfg->algo : RADON_ALGO_AUTO;
    return algo == RADON_ALGO_AUTO && batch == 1 &&
           (cfg == nullptr || (cfg->views_per_cta == 0 && cfg->rows_per_slab == 0 && cfg->images_per_cta == 0 &&
                               cfg->tile == 0 && cfg->threads == 0));
}

radon_status project(const radon_geometry* g, const void* in, void* out, radon_dtype dt, int batch,
                     const radon_launch_config* cfg, void* stream, bool forward, void* ws, size_t ws_bytes,
                     const radon_epilogue* epi) {
    radon_status st = validate_call(g, in, out, dt, batch);
    if (st != RADON_OK) return st;
    st = validate_epilogue(epi, dt);
    if (st != RADON_OK) return st;
    const Epilogue ep = epi ? Epilogue{epi->op_scale, epi->op_scale_dev, epi->add_scale, epi->add}
                            : identity_epilogue();
    const int algo = cfg ? cfg->algo : RADON_ALGO_AUTO;
    if (algo != RADON_ALGO_AUTO && algo != RADON_ALGO_PLAIN && algo != RADON_ALGO_TILED)
        return fail(RADON_ERR_INVALID_ARG, "unknown algo");
    if (cfg != nullptr && cfg->weights != RADON_WEIGHTS_DEFAULT && cfg->weights != RADON_WEIGHTS_F32 &&
        cfg->weights != RADON_WEIGHTS_F16)
        return fail(RADON_ERR_INVALID_ARG,
                    "weights must be 0 or 1 (FP32 weights) or 2 (FP16 weights, FP16 storage only)");
    const int threads = cfg ? cfg->threads : 0;
    if (threads < 0 || threads > 1024 || (threads % 32) != 0)
        return fail(RADON_ERR_INVALID_ARG, "threads must be 0 or a multiple of 32 up to 1024");
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (batch == 0) return RADON_OK;
    st = check_device(g);
    if (st != RADON_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int images = cfg ? cfg->images_per_cta : 0;
    // One image under AUTO with no tile parameters: the single-image kernels (a batch-interleaved
    // group would carry the image in one of its 4 / 8 / 16 slots).  The forward needs its quad
    // texels in the workspace; without one it continues below.
    const bool single = single_image_call(cfg, batch);
    if (single && !forward) {
        std::string why;
        st = launch_backward_single(g, in, out, dt, ep, s, &why);
        if (st == RADON_OK) return RADON_OK;
        if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
    }
    if (single && forward && ws != nullptr && ws_bytes >= single_forward_workspace_bytes(g, dt)) {
        st = launch_forward_single(g, in, out, dt, ws, ep, s);
        if (st != RADON_OK) return st;
        return RADON_OK;
    }
    if (!forward && algo != RADON_ALGO_PLAIN && ws != nullptr) {
        // Packed path: pack the sinogram batch once, then copy detector windows straight into
        // shared memory.  A too small workspace or a geometry the kernel refuses continues below.
        const int bg = backward_packed_images_per_cta(g, batch, dt, cfg);
        if (ws_bytes >= packed_sino_bytes(g->V, g->D, batch, bg, dt)) {
            cudaError_t e = launch_pack_sino(in, ws, g->V, g->D, batch, bg, dt, s);
            if (e != cudaSuccess) return cuda_fail(e, "sinogram pack launch");
            std::string why;
            count_launches(1);
            st = launch_backward_packed(g, ws, out, dt, batch, bg, ep, s, &why);
            if (st == RADON_OK) {
                count_launches(1);
                return RADON_OK;
            }
            if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
        }
    }
    if (!forward && algo != RADON_ALGO_PLAIN) {
        std::string why;
        st = launch_backward_tiled(g, in, out, dt, batch, images, ep, s, &why);
        if (st == RADON_OK) {
            count_launches(1);
            return RADON_OK;
        }
        if (st != RADON_ERR_UNSUPPORTED || algo == RADON_ALGO_TILED) return fail(st, why);
        // AUTO: this geometry / buffer does not fit the tiled kernel; the plain kernel serves it
    }
    if (forward && algo != RADON_ALGO_PLAIN && ws != nullptr && ws_bytes >= packed_image_bytes(g->n, batch, dt)) {
        // Packed path: pack the batch once, then copy bands of texels straight into shared memory.
        // one lane per ray first; where no one-lane shape fits and the caller left the shape to the
        // library, two lanes (half the detectors per CTA: narrower bands).  An explicit views per
        // CTA keeps one lane per ray.
        const bool fixed = cfg != nullptr && cfg->views_per_cta != 0;
        std::string why;
        bool packed_done = false;
        for (int lanes = 1; lanes <= (fixed ? 1 : 2); ++lanes) {
            for (int i = 0; i < (fixed ? 1 : 4); ++i) {
                const radon_launch_config c = packed_forward_config(cfg, dt, i);
                if (!packed_done) {
                    cudaError_t e = launch_pack_images(in, ws, g->n, batch, dt, s);
                    if (e != cudaSuccess) return cuda_fail(e, "pack launch");
                    count_launches(1);
                    packed_done = true;
                }
                st = launch_forward_packed(const_cast<radon_geometry*>(g), ws, out, dt, batch, &c, ep, s, &why,
                                           lanes);
                if (st == RADON_OK) {
                    count_launches(1);
                    return RADON_OK;
                }
                if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
            }
        }
        // no packed shape fits: continue with the paths that need no workspace
    }
    if (forward && algo != RADON_ALGO_PLAIN) {
        // An explicit views-per-CTA is used as given.  Otherwise the shapes are tried in order of
        // preference: a sparse view set or a wide fan may need fewer views (or more, narrower
        // detector ranges) for the working band to fit one TMA box.
        static const int kViews[4] = {8, 4, 2, 1};
        const bool fixed = cfg != nullptr && cfg->views_per_cta != 0;
        std::string why;
        for (int i = 0; i < (fixed ? 1 : 4); ++i) {
            radon_launch_config c = {RADON_ALGO_TILED, fixed ? cfg->views_per_cta : kViews[i],
                                     cfg ? cfg->rows_per_slab : 0, 0, 0, 0, cfg ? cfg->weights : 0};
            st = launch_forward_tiled(const_cast<radon_geometry*>(g), in, out, dt, batch, &c, ep, s, &why);
            if (st == RADON_OK) {
                count_launches(1);
                return RADON_OK;
            }
            if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
        }
        if (algo == RADON_ALGO_TILED) return fail(st, why);
        // AUTO: no tiled shape fits this geometry / buffer; the plain kernel serves it
    }
    cudaError_t e;
    if (forward) {
        e = launch_forward_plain(g, in, out, dt, batch, threads, ep, s);
    } else {
        e = launch_backward_plain(g, in, out, dt, batch, threads, ep, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, forward ? "forward launch" : "backward launch");
    count_launches(1);
    return RADON_OK;
}

}  // namespace radon

using namespace radon;

extern "C" {

radon_status radon_geometry_create_parallel(int n, const double* angles, int n_angles, int det_count,
                                            double det_spacing, double step, radon_geometry** out) {
    return create_common(n, angles, n_angles, det_count, det_spacing, step, 0, 0.0, 0.0, 0, out);
}

radon_status radon_geometry_create_fanbeam(int n, const double* angles, int n_angles, double source_distance,
                                           double det_distance, int det_count, double det_spacing, double step,
                                           radon_geometry** out) {
    return create_common(n, angles, n_angles, det_count, det_spacing, step, 1, source_distance, det_distance, 0, out);
}

radon_status radon_geometry_create(const radon_geometry_desc* desc, radon_geometry** out) {
    if (desc == nullptr) return fail(RADON_ERR_INVALID_ARG, "desc is NULL");
    if (desc->is_fan != 0 && desc->is_fan != 1) return fail(RADON_ERR_INVALID_ARG, "is_fan must be 0 or 1");
    return create_common(desc->n, desc->angles, desc->n_angles, desc->det_count, desc->det_spacing, desc->step,
                         desc->is_fan, desc->source_distance, desc->det_distance, desc->host_only, out);
}

radon_status radon_geometry_copy_rays(const radon_geometry* g, float* rays, int32_t* counts) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    const size_t nr = (size_t)g->V * g->D;
    if (rays != nullptr) {
        for (size_t r = 0; r < nr; ++r) {
            const RayT& t = g->h_ray[r];
            float* o = rays + 8 * r;
            o[0] = (float)t.J0;
            o[1] = (float)t.I0;
            o[2] = t.fx0;
            o[3] = t.fy0;
            o[4] = t.dxh;
            o[5] = t.dyh;
            o[6] = t.dxl;
            o[7] = t.dyl;
        }
    }
    if (counts != nullptr) std::memcpy(counts, g->h_nk.data(), nr * sizeof(int));
    return RADON_OK;
}

void radon_geometry_destroy(radon_geometry* geometry) {
    if (geometry == nullptr || geometry->magic != kGeometryMagic) return;
    release(geometry);
}

radon_status radon_geometry_adjoint_table_size(const radon_geometry* g, size_t* bytes) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (bytes == nullptr) return fail(RADON_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = adjoint_table_bytes(g);
    return RADON_OK;
}

radon_status radon_geometry_build_adjoint_table(radon_geometry* g) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (g->host_only) return fail(RADON_ERR_INVALID_ARG, "host-only geometry");
    st = check_device(g);
    if (st != RADON_OK) return st;
    std::string why;
    st = build_adjoint_table(g, &why);
    if (st != RADON_OK) return fail(st, why);
    return RADON_OK;
}

radon_status radon_geometry_adjoint_table_overflow(const radon_geometry* g, double* fraction) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (fraction == nullptr) return fail(RADON_ERR_INVALID_ARG, "fraction is NULL");
    *fraction = g->d_tab_w != nullptr ? g->tab_overflow : 0.0;
    return RADON_OK;
}

radon_status radon_geometry_free_adjoint_table(radon_geometry* g) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    free_adjoint_table(g);
    return RADON_OK;
}

radon_status radon_geometry_get_info(const radon_geometry* g, radon_geometry_info* out) {
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (out == nullptr) return fail(RADON_ERR_INVALID_ARG, "out is NULL");
    out->n = g->n;
    out->n_angles = g->V;
    out->det_count = g->D;
    out->is_fan = g->fan;
    out->det_spacing = g->ds;
    out->step = g->h;
    out->source_distance = g->S;
    out->det_distance = g->Ddet;
    out->sample_count = g->samples;
    out->device = g->device;
    return RADON_OK;
}

int64_t radon_geometry_sample_count(const radon_geometry* g) {
    if (validate_geometry(g) != RADON_OK) return -1;
    return g->samples;
}

radon_status radon_forward(const radon_geometry* g, const void* img, void* sino, radon_dtype dtype, int batch,
                           void* stream) {
    return project(g, img, sino, dtype, batch, nullptr, stream, true, nullptr, 0, nullptr);
}

radon_status radon_backward(const radon_geometry* g, const void* sino, void* img, radon_dtype dtype, int batch,
                            void* stream) {
    return project(g, sino, img, dtype, batch, nullptr, stream, false, nullptr, 0, nullptr);
}

radon_status radon_forward_ex(const radon_geometry* g, const void* img, void* sino, radon_dtype dtype, int batch,
                              const radon_launch_config* config, void* stream) {
    return project(g, img, sino, dtype, batch, config, stream, true, nullptr, 0, nullptr);
}

radon_status radon_backward_ex(const radon_geometry* g, const void* sino, void* img, radon_dtype dtype, int batch,
                               const radon_launch_config* config, void* stream) {
    return project(g, sino, img, dtype, batch, config, stream, false, nullptr, 0, nullptr);
}

size_t radon_forward_workspace_size(const radon_geometry* g, radon_dtype dtype, int batch) {
    if (validate_geometry(g) != RADON_OK) return 0;
    if (dtype != RADON_F32 && dtype != RADON_F16 && dtype != RADON_BF16) return 0;
    if (batch < 0) return 0;
    // a single image runs the single-image forward, whose quad texels carry a one-pixel border
    if (batch == 1) return std::max(packed_image_bytes(g->n, batch, dtype), single_forward_workspace_bytes(g, dtype));
    return packed_image_bytes(g->n, batch, dtype);
}

radon_status radon_forward_images_per_cta(const radon_geometry* g, radon_dtype dtype, int batch,
                                          const radon_launch_config* config, int* images) {
    if (images == nullptr) return fail(RADON_ERR_INVALID_ARG, "images is NULL");
    *images = 0;
    radon_status st = validate_geometry(g);
    if (st != RADON_OK) return st;
    if (dtype != RADON_F32 && dtype != RADON_F16 && dtype != RADON_BF16) return fail(RADON_ERR_INVALID_ARG, "unknown dtype");
    if (batch < 0) return fail(RADON_ERR_INVALID_ARG, "batch must be >= 0");
    const int algo = config ? config->algo : RADON_ALGO_AUTO;
    if (batch == 0 || algo == RADON_ALGO_PLAIN || single_image_call(config, batch)) return RADON_OK;
    const bool f16w = dtype == RADON_F16 && config != nullptr && config->weights == RADON_WEIGHTS_F16;
    const bool fixed = config != nullptr && config->views_per_cta != 0;
    for (int lanes = 1; lanes <= (fixed ? 1 : 2); ++lanes) {
        for (int i = 0; i < (fixed ? 1 : 4); ++i) {
            const radon_launch_config c = packed_forward_config(config, dtype, i);
            PackedFwdShape sh;
            std::string why;
            if (packed_forward_shape(const_cast<radon_geometry*>(g), dtype, batch, &c, f16w, lanes, &sh, &why) ==
                RADON_OK) {
                *images = sh.NG * (dtype == RADON_F32 ? 4 : 8);
                return RADON_OK;
            }
        }
    }
    return RADON_OK;
}

radon_status radon_forward_ws(const radon_geometry* g, const void* img, void* sino, radon_dtype dtype, int batch,
                              const radon_launch_config* config, void* workspace, size_t workspace_bytes,
                              void* stream) {
    if (workspace != nullptr && ((uintptr_t)workspace & 15) != 0)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    return project(g, img, sino, dtype, batch, config, stream, true, workspace, workspace_bytes, nullptr);
}

size_t radon_backward_workspace_size(const radon_geometry* g, radon_dtype dtype, int batch) {
    if (validate_geometry(g) != RADON_OK) return 0;
    if (dtype != RADON_F32 && dtype != RADON_F16 && dtype != RADON_BF16) return 0;
    if (batch < 0) return 0;
    return packed_sino_bytes(g->V, g->D, batch, backward_packed_images_per_cta(g, batch, dtype, nullptr), dtype);
}

radon_status radon_backward_ws(const radon_geometry* g, const void* sino, void* img, radon_dtype dtype, int batch,
                               const radon_launch_config* config, void* workspace, size_t workspace_bytes,
                               void* stream) {
    if (workspace != nullptr && ((uintptr_t)workspace & 15) != 0)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    return project(g, sino, img, dtype, batch, config, stream, false, workspace, workspace_bytes, nullptr);
}

radon_status radon_forward_fused(const radon_geometry* g, const void* img, void* sino, radon_dtype dtype, int batch,
                                 const radon_epilogue* epilogue, const radon_launch_config* config, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    if (workspace != nullptr && ((uintptr_t)workspace & 15) != 0)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    return project(g, img, sino, dtype, batch, config, stream, true, workspace, workspace_bytes, epilogue);
}

radon_status radon_backward_fused(const radon_geometry* g, const void* sino, void* img, radon_dtype dtype, int batch,
                                  const radon_epilogue* epilogue, const radon_launch_config* config, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    if (workspace != nullptr && ((uintptr_t)workspace & 15) != 0)
        return fail(RADON_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    return project(g, sino, img, dtype, batch, config, stream, false, workspace, workspace_bytes, epilogue);
}

uint64_t radon_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

radon_status radon_get_device_error(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int word = 0;
    e = read_and_clear_device_error(&word);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (word == RADON_ERR_TIMEOUT) return fail(RADON_ERR_TIMEOUT, "a kernel's bounded wait expired");
    if (word == RADON_ERR_DEVICE_BOUNDS) return fail(RADON_ERR_DEVICE_BOUNDS, "a kernel's bounds check fired");
    if (word != 0) return fail(RADON_ERR_CUDA, "unknown device error code " + std::to_string(word));
    return RADON_OK;
}

const char* radon_status_string(radon_status status) {
    switch (status) {
        case RADON_OK: return "RADON_OK";
        case RADON_ERR_INVALID_ARG: return "RADON_ERR_INVALID_ARG";
        case RADON_ERR_UNSUPPORTED: return "RADON_ERR_UNSUPPORTED";
        case RADON_ERR_OOM: return "RADON_ERR_OOM";
        case RADON_ERR_CUDA: return "RADON_ERR_CUDA";
        case RADON_ERR_TIMEOUT: return "RADON_ERR_TIMEOUT";
        case RADON_ERR_DEVICE_BOUNDS: return "RADON_ERR_DEVICE_BOUNDS";
    }
    return "RADON_ERR_UNKNOWN";
}

const char* radon_last_error_message(void) { return g_last_error.c_str(); }

int radon_abi_version(void) { return RADON_ABI_VERSION; }

}  // extern "C"
