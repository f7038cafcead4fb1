// Instantiations of the packed adjoint's launcher for __nv_bfloat16 storage (one translation unit per storage
// type, so the kernels compile in parallel).
#include "backward_packed.cuh"

namespace radon {

template radon_status launch_backward_packed_t<__nv_bfloat16, 8>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                        const Epilogue&, cudaStream_t, std::string*,
                                                        const CUtensorMap&, uint32_t, int*);
template radon_status launch_backward_packed_t<__nv_bfloat16, 16>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                         const Epilogue&, cudaStream_t, std::string*,
                                                         const CUtensorMap&, uint32_t, int*);
template radon_status launch_backward_packed_t<__nv_bfloat16, 32>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                         const Epilogue&, cudaStream_t, std::string*,
                                                         const CUtensorMap&, uint32_t, int*);

}  // namespace radon
