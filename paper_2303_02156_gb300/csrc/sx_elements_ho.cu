// sx_elements_ho.cu -- instantiations of the element kernel with the
// high-order tets compiled in (KINDS 64: high-order tets only; 127: every
// stencil kind), and the high-order tets' per-point phase.
#include <cuda_runtime.h>

#include <algorithm>

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

cudaError_t launch_tetho_points(const ElemLaunch& L, int scene, int blk, int64_t n_el, int nq,
                                cudaStream_t s)
{
    const int64_t n = n_el * nq;
    if (!n) return cudaSuccess;
    const unsigned g = (unsigned)((n + 127) / 128);
    if (L.precision == SX_FP32) k_tetho_points<float><<<g, 128, 0, s>>>(L, scene, blk);
    else k_tetho_points<double><<<g, 128, 0, s>>>(L, scene, blk);
    return cudaGetLastError();
}

int tetho_block_smem(int K, int nq) { return tetho_smem_bytes(K, nq, true, 8); }

cudaError_t launch_tetho_blocks(const ElemLaunch& L, int scene, int blk, int64_t n_el, int K,
                                int nq, cudaStream_t s)
{
    if (!n_el) return cudaSuccess;
    const bool proj = L.level >= 2 && L.project;
    // elements per block: as many as the owned blocks, gradients and energy
    // of each leave threads for (small K), at most 8
    const int items = K * (K + 1) / 2 + K + 1;
    const int epc = std::max(1, std::min(8, kHoBlockThreads / items));
    const bool f32 = L.precision == SX_FP32;
    const int smem = epc * tetho_smem_bytes(K, nq, proj, f32 ? 4 : 8);
    const unsigned g = (unsigned)((n_el + epc - 1) / epc);
    const void* fn = f32 ? (const void*)k_tetho_blocks<float, float>
                         : (const void*)k_tetho_blocks<double, double>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    if (f32) k_tetho_blocks<float, float><<<g, kHoBlockThreads, smem, s>>>(L, scene, blk, epc);
    else k_tetho_blocks<double, double><<<g, kHoBlockThreads, smem, s>>>(L, scene, blk, epc);
    return cudaGetLastError();
}

}  // namespace sx
