// Instantiations of the packed adjoint's launcher for float storage (one translation unit per storage
// type, so the kernels compile in parallel).
#include "backward_packed.cuh"

namespace radon {

template radon_status launch_backward_packed_t<float, 8>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                        const Epilogue&, cudaStream_t, std::string*,
                                                        const CUtensorMap&, uint32_t, int*);
template radon_status launch_backward_packed_t<float, 16>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                         const Epilogue&, cudaStream_t, std::string*,
                                                         const CUtensorMap&, uint32_t, int*);
template radon_status launch_backward_packed_t<float, 32>(const radon_geometry*, const void*, void*, radon_dtype, int, int,
                                                         const Epilogue&, cudaStream_t, std::string*,
                                                         const CUtensorMap&, uint32_t, int*);

}  // namespace radon
