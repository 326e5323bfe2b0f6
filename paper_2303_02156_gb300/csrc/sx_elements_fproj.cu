// sx_elements_fproj.cu -- instantiations of the element kernel with
// the F-space (material) projection of SNH tets compiled in (KINDS 9: SNH
// tets only; 15: every stencil kind).
#include <cuda_runtime.h>

#include "sx_elements.cuh"

namespace sx {

const void* elements_kernel_fproj(int kinds, bool f32)
{
    return kinds == 9 ? elements_kernel_ptr<9>(f32) : elements_kernel_ptr<15>(f32);
}

cudaError_t launch_elements_fproj(int kinds, bool f32, const ElemLaunch& L, int grid,
                                 cudaStream_t s)
{
    if (kinds == 9) elements_launch<9>(f32, L, grid, s);
    else elements_launch<15>(f32, L, grid, s);
    return cudaGetLastError();
}

}  // namespace sx
