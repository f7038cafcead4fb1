// Forward projection for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all, or not at the moment they project: a real-time or
// safety-certified loop that forbids allocation after start-up, code that must not let an
// allocation synchronise the device in the middle of its stream work, or a plain C host that has
// no device allocator and no caching pool to borrow a workspace from.  radon_forward_static_scratch
// gives them the packed forward path -- the one that needs a scratch workspace for the packed
// image batch -- with that scratch in a fixed, file-scope device array instead: nothing is
// allocated, by this library or by anyone else, at any call.
//
// Costs and rules of the shared array (kStaticScratchBytes, 32 MiB):
//   * every GPU that loads the library holds the array until the process exits;
//   * a call needs the packed batch, 2 * ceil(batch / BG) * N^2 * 16 bytes (BG = 4 images per texel
//     for FP32 storage, 8 for 16-bit; a batch of one is one group); larger requests are rejected
//     with RADON_ERR_INVALID_ARG (split the batch);
//   * every call packs its whole batch into the array and so overwrites what the previous call left
//     there; nothing in it has to start at zero (the packing writes every texel the kernel reads,
//     padding included);
//   * calls whose work overlaps on the GPU (two streams, or a second call before the first one's
//     kernels have run on another stream) race on the array and must be ordered by the caller;
//   * the first call on each device looks up the array's device address with that device current
//     (cudaGetSymbolAddress) and keeps it for the life of the process; make that first call before
//     any stream capture starts.  The kept address is not valid across a reset of the device's
//     primary context (cudaDeviceReset): do not call this entry point after one.
#include <mutex>

#include "radon_internal.h"

namespace radon {

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

// Device address of the array for the current device (looked up once per device).
radon_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(RADON_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RADON_OK;
}

}  // namespace

}  // namespace radon

using namespace radon;

extern "C" RADON_API radon_status radon_forward_static_scratch(const radon_geometry* geometry, const void* img,
                                                               void* sino, radon_dtype dtype, int batch,
                                                               void* stream) {
    radon_status st = validate_call(geometry, img, sino, dtype, batch);
    if (st != RADON_OK) return st;
    if (geometry->host_only) return fail(RADON_ERR_INVALID_ARG, "geometry was created host-only; it cannot launch");
    if (batch == 0) return RADON_OK;
    const size_t need = packed_image_bytes(geometry->n, batch, dtype);
    if (need > kStaticScratchBytes)
        return fail(RADON_ERR_INVALID_ARG, "this batch needs " + std::to_string(need) +
                                               " bytes of scratch; the static scratch holds " +
                                               std::to_string(kStaticScratchBytes) + " bytes (split the batch)");
    st = check_device(geometry);
    if (st != RADON_OK) return st;
    void* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != RADON_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_pack_images(img, scratch, geometry->n, batch, dtype, s);
    if (e != cudaSuccess) return cuda_fail(e, "pack launch");
    count_launches(1);
    static const int kViews[4] = {8, 4, 2, 1};
    std::string why;
    for (int lanes = 1; lanes <= 2; ++lanes) {
        for (int i = 0; i < 4; ++i) {
            radon_launch_config c = {RADON_ALGO_TILED, kViews[i], 0, 0, 0, 0, 0};
            st = launch_forward_packed(const_cast<radon_geometry*>(geometry), scratch, sino, dtype, batch, &c,
                                       identity_epilogue(), s, &why, lanes);
            if (st == RADON_OK) {
                count_launches(1);
                return RADON_OK;
            }
            if (st != RADON_ERR_UNSUPPORTED) return fail(st, why);
        }
    }
    // No packed shape fits this geometry: the paths that need no scratch at all serve it.
    return radon_forward(geometry, img, sino, dtype, batch, stream);
}
