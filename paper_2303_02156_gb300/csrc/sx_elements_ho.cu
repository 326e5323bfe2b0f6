// sx_elements_ho.cu -- instantiations of the element kernel with the
// high-order tets compiled in (KINDS 64: high-order tets only; 127: every
// stencil kind).
#include <cuda_runtime.h>

#include "sx_elements.cuh"

namespace sx {

const void* elements_kernel_ho(int kinds, bool f32)
{
    return kinds == 64 ? elements_kernel_ptr<64>(f32) : elements_kernel_ptr<127>(f32);
}

cudaError_t launch_elements_ho(int kinds, bool f32, const ElemLaunch& L, int grid, cudaStream_t s)
{
    if (kinds == 64) elements_launch<64>(f32, L, grid, s);
    else elements_launch<127>(f32, L, grid, s);
    return cudaGetLastError();
}

}  // namespace sx
