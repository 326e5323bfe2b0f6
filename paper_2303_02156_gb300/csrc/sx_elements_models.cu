// sx_elements_models.cu -- instantiations of the element kernel with
// tets of every density (NH, StVK, co-rotational, ARAP besides SNH,
// with the material projection of the SNH tets; KINDS 25: tets only; 63:
// every stencil kind, friction included).
#include <cuda_runtime.h>

#include "sx_elements.cuh"

namespace sx {

const void* elements_kernel_models(int kinds, bool f32)
{
    return kinds == 25 ? elements_kernel_ptr<25>(f32) : elements_kernel_ptr<63>(f32);
}

cudaError_t launch_elements_models(int kinds, bool f32, const ElemLaunch& L, int grid,
                                 cudaStream_t s)
{
    if (kinds == 25) elements_launch<25>(f32, L, grid, s);
    else elements_launch<63>(f32, L, grid, s);
    return cudaGetLastError();
}

}  // namespace sx
