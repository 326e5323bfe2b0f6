// sx_assemble.cu -- global assembly (§5.3, Eq. 11; Algorithm 1 block
// insertion) and the inertia term of the incremental potential (§3,
// Eq. 2), without atomics.
//
// The paper inserts each element block into the BCRS matrix under a
// mutex. Here each BSR block instead gathers its contributions: the
// finalize step built, for every block, the element-id-ordered list of
// (stencil, local a, local b) that land on it, so the sum is formed in a
// fixed order by one thread and written once. The gradient is gathered the
// same way per node. Inertia adds m/dt^2 I to the diagonal blocks after the
// element terms, and m/dt^2 (x - x_tilde) to the gradient.
#include <cuda_runtime.h>

#include "sx_internal.cuh"

namespace sx {

static constexpr int kAsmThreads = 256;

// one thread per BSR block; AT is the accumulation type (double in the FP64
// form; float in the FP32 form, whose element blocks and stored values are
// float: on this part a float-to-double conversion costs an FP64 slot)
template <typename HT, typename VT, typename AT>
__global__ void __launch_bounds__(kAsmThreads)
k_assemble_vals(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const int ti = blockIdx.x;
    if (ti >= ntiles) return;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (S.sc && !S.sc->active) return;
    if ((int)threadIdx.x >= T.count) return;
    // the tile's blocks in ascending order of list length (a permutation
    // within the tile), so that a warp's lists have similar lengths
    const int64_t slot = S.slot_order[T.start + threadIdx.x];
    const HT* He = (const HT*)S.He;
    AT acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = AT(0);
    const int b = S.slot_ptr[slot], e = S.slot_ptr[slot + 1];
    for (int k = b; k < e; ++k) {
        const int code = S.slot_src[k];
        const int64_t st = code >> 4;
        const int la = (code >> 2) & 3, lb = code & 3;
        const HT* blk;
        if (la <= lb) {
            blk = He + 90 * st + 9 * up_index(la, lb);
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] += (AT)blk[q];
        } else {
            blk = He + 90 * st + 9 * up_index(lb, la);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[i * 3 + j] += (AT)blk[j * 3 + i];
        }
    }
    VT* out = (sizeof(VT) == 8) ? (VT*)S.vals64 : (VT*)S.vals32;
#pragma unroll
    for (int q = 0; q < 9; ++q) out[9 * slot + q] = (VT)acc[q];
}

// inertia on the diagonal blocks, after the element terms
template <typename VT>
__global__ void k_inertia_diag(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const int ti = blockIdx.x;
    if (ti >= ntiles) return;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (S.sc && !S.sc->active) return;
    if (!S.inertia_on) return;
    if ((int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
    VT* out = (sizeof(VT) == 8) ? (VT*)S.vals64 : (VT*)S.vals32;
    const int64_t d = S.diag_slot[n];
    const double h = S.mass[n] * S.inv_dt2;
    out[9 * d + 0] = (VT)((double)out[9 * d + 0] + h);
    out[9 * d + 4] = (VT)((double)out[9 * d + 4] + h);
    out[9 * d + 8] = (VT)((double)out[9 * d + 8] + h);
}

cudaError_t launch_assemble_vals(const AsmLaunch& L, cudaStream_t s)
{
    if (L.ntiles == 0) return cudaSuccess;
    if (L.precision == SX_FP32)
        k_assemble_vals<float, float, float><<<L.ntiles, kAsmThreads, 0, s>>>(L.scenes, L.tiles,
                                                                            L.ntiles);
    else
        k_assemble_vals<double, double, double><<<L.ntiles, kAsmThreads, 0, s>>>(
            L.scenes, L.tiles, L.ntiles);
    return cudaGetLastError();
}

cudaError_t launch_inertia_diag(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                int precision, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    if (precision == SX_FP32)
        k_inertia_diag<float><<<ntiles, kAsmThreads, 0, s>>>(scenes, node_tiles, ntiles);
    else
        k_inertia_diag<double><<<ntiles, kAsmThreads, 0, s>>>(scenes, node_tiles, ntiles);
    return cudaGetLastError();
}

// per node: grad = sum of element gradients (element order) + inertia;
// tile partials: [0] inertia energy, [1] ||g_free||^2
__global__ void __launch_bounds__(kAsmThreads)
k_assemble_grad(const SceneDev* scenes, const Tile* tiles, int ntiles, int with_grad,
                double* part)
{
    __shared__ double sh[2][kAsmThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    double ein = 0.0, gn = 0.0;
    const bool live = !(S.sc && !S.sc->active);
    if (live && (int)threadIdx.x < T.count) {
        const int64_t n = T.start + threadIdx.x;
        double r[3] = {0.0, 0.0, 0.0};
        if (S.inertia_on) {
            const double h = S.mass[n] * S.inv_dt2;
            const double dt = S.dt;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                // in a Newton step the residual is formed from the step's
                // increments: x - x_start is exact for nearby values, which
                // keeps E_BE above rounding for the last Newton decreases
                r[i] = S.inertia_mode
                           ? (S.x[3 * n + i] - S.x_start[3 * n + i]) -
                                 (dt * S.v[3 * n + i] + dt * dt * S.sc->grav[i])
                           : S.x[3 * n + i] - S.x_tilde[3 * n + i];
                ein += r[i] * r[i];
                r[i] *= h;
            }
            ein *= 0.5 * h;
        }
        if (with_grad) {
            double g[3] = {0.0, 0.0, 0.0};
            const int b = S.node_ptr[n], e = S.node_ptr[n + 1];
            for (int k = b; k < e; ++k) {
                const int code = S.node_src[k];
                const double* src = S.ge + 12 * (int64_t)(code >> 2) + 3 * (code & 3);
                g[0] += src[0];
                g[1] += src[1];
                g[2] += src[2];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                g[i] += r[i];
                S.grad[3 * n + i] = g[i];
            }
            if (!S.pinned[n]) gn = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        }
    }
    sh[0][threadIdx.x] = ein;
    sh[1][threadIdx.x] = gn;
    __syncthreads();
    for (int w = kAsmThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * ti + 0] = sh[0][0];
        part[2 * ti + 1] = sh[1][0];
    }
}

cudaError_t launch_assemble_grad(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                 double* tile_part, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    k_assemble_grad<<<ntiles, kAsmThreads, 0, s>>>(scenes, node_tiles, ntiles, 1, tile_part);
    return cudaGetLastError();
}

cudaError_t launch_inertia_energy(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                  const double* unused, double* tile_part, int use_trial,
                                  cudaStream_t s)
{
    (void)unused;
    (void)use_trial;
    if (ntiles == 0) return cudaSuccess;
    k_assemble_grad<<<ntiles, kAsmThreads, 0, s>>>(scenes, node_tiles, ntiles, 0, tile_part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ reductions
static constexpr int kRedThreads = 256;

__device__ __forceinline__ double* scal_field(SceneScal* sc, int f)
{
    switch (f) {
        case F_E: return &sc->E;
        case F_GNORM2: return &sc->gnorm2;
        case F_FEXT2: return &sc->fext2;
        default: return &sc->gdx;
    }
}

// one block per scene; fixed partition and tree => deterministic
__global__ void k_scene_reduce(const double* part, int stride, int off, const int* tbeg,
                               const int* tend, const SceneDev* scenes, int field,
                               int accumulate)
{
    __shared__ double sh[kRedThreads];
    const int s = blockIdx.x;
    SceneScal* sc = scenes[s].sc;
    const int b = tbeg[s], e = tend[s];
    double acc = 0.0;
    for (int t = b + threadIdx.x; t < e; t += kRedThreads) acc += part[(int64_t)t * stride + off];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && sc->active) {
        double* dst = scal_field(sc, field);
        *dst = accumulate ? *dst + sh[0] : sh[0];
    }
}

cudaError_t launch_scene_reduce(const double* part, int stride, int off, const int* tbeg,
                                const int* tend, int nscenes, const SceneDev* scenes,
                                int field, int accumulate, cudaStream_t s)
{
    if (nscenes == 0) return cudaSuccess;
    k_scene_reduce<<<nscenes, kRedThreads, 0, s>>>(part, stride, off, tbeg, tend, scenes, field,
                                                   accumulate);
    return cudaGetLastError();
}

// integer counters per element tile: barrier d <= 0, non-finite, projected
__global__ void k_scene_reduce_int(const int* bad, const int* nonfin, const int* clamped,
                                   const int* tbeg, const int* tend, const SceneDev* scenes)
{
    __shared__ int sh[3][kRedThreads];
    const int s = blockIdx.x;
    SceneScal* sc = scenes[s].sc;
    int a = 0, c = 0, p = 0;
    for (int t = tbeg[s] + threadIdx.x; t < tend[s]; t += kRedThreads) {
        a += bad[t];
        c += nonfin[t];
        p += clamped[t];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = c;
    sh[2][threadIdx.x] = p;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && sc->active) {
        sc->bad_state = sh[0][0];
        sc->nonfinite = sh[1][0] + sc->clamp_fail;
        sc->clamp_fail = 0;
        sc->clamped = sh[2][0];
    }
}

cudaError_t launch_scene_reduce_flags(const int* bad, const int* nonfin, const int* clamped,
                                      const int* tbeg, const int* tend, int nscenes,
                                      const SceneDev* scenes, cudaStream_t s)
{
    if (nscenes == 0) return cudaSuccess;
    k_scene_reduce_int<<<nscenes, kRedThreads, 0, s>>>(bad, nonfin, clamped, tbeg, tend,
                                                       scenes);
    return cudaGetLastError();
}

// copy every scene's scalars into one array (for a single readback)
__global__ void k_gather_scal(const SceneDev* scenes, int n, SceneScal* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *scenes[i].sc;
}

cudaError_t launch_gather_scal(const SceneDev* scenes, int n, SceneScal* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_gather_scal<<<(n + 127) / 128, 128, 0, s>>>(scenes, n, out);
    return cudaGetLastError();
}

// write per-scene control values: active flags and (optionally) step sizes
__global__ void k_set_scal(const SceneDev* scenes, int n, const int* active,
                           const double* ls_alpha, const double* pcg_tol)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    SceneScal* sc = scenes[i].sc;
    if (active) sc->active = active[i];
    if (ls_alpha) sc->ls_alpha = ls_alpha[i];
    if (pcg_tol) sc->pcg_tol = pcg_tol[i];
}

cudaError_t launch_set_scal(const SceneDev* scenes, int n, const int* active,
                            const double* ls_alpha, const double* pcg_tol, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_set_scal<<<(n + 127) / 128, 128, 0, s>>>(scenes, n, active, ls_alpha, pcg_tol);
    return cudaGetLastError();
}

}  // namespace sx
