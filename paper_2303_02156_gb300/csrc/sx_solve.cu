// sx_solve.cu -- the backward-Euler Newton step's vector kernels (§3,
// Eqs. 2-3) and the 3x3 block-Jacobi preconditioned CG of §7.2, batched
// over scenes with per-scene scalars on the device.
//
// PCG iteration (per scene, x0 = 0, b = -g on free DOFs, 0 on pinned):
//   p_new = z + beta p_old;  q = A p_new;  alpha = (r.z) / (p_new.q)
//   dx += alpha p_new;  r -= alpha q;  z = Minv r
//   stop when ||r|| <= tol ||b||;  beta = r.z_new / r.z
// The direction update is fused into the SpMV (p_old and p_new alternate
// between two buffers), so an iteration is two vector kernels and two
// one-block-per-scene reductions that also form alpha and beta. Pinned
// DOFs are eliminated by mask: their rows are identity and their columns
// are skipped.
#include <cuda_runtime.h>

#include "sx_internal.cuh"

namespace sx {

static constexpr int kVecThreads = 256;
static constexpr int kRedT = 256;

__device__ __forceinline__ bool scene_live(const SceneDev& S)
{
    return S.sc == nullptr || S.sc->active;
}

// ------------------------------------------------------------------ predictor
// x_start = x, x~ = x + dt v + dt^2 g; tile partial: sum over free nodes of
// m^2 |g|^2 (the external-force scale of the Newton residual test)
__global__ void __launch_bounds__(kVecThreads)
k_predict(const SceneDev* scenes, const Tile* tiles, int ntiles, double* part)
{
    __shared__ double sh[kVecThreads];
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    double f2 = 0.0;
    if (scene_live(S) && (int)threadIdx.x < T.count) {
        const int64_t n = T.start + threadIdx.x;
        const double dt = S.dt;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double x = S.x[3 * n + i];
            const double g = S.sc->grav[i];
            S.x_start[3 * n + i] = x;
            S.x_tilde[3 * n + i] = x + dt * S.v[3 * n + i] + dt * dt * g;
            if (!S.pinned[n]) f2 += S.mass[n] * S.mass[n] * g * g;
        }
    }
    sh[threadIdx.x] = f2;
    __syncthreads();
    for (int w = kVecThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

cudaError_t launch_predict(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                           double* part, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_predict<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PCG setup
template <typename VT>
__device__ __forceinline__ void inv3x3(const VT* A, double* Ai)
{
    double a[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = (double)A[k];
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    double id = 1.0 / det;
    Ai[0] = c00 * id;
    Ai[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    Ai[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    Ai[3] = c01 * id;
    Ai[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    Ai[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    Ai[6] = c02 * id;
    Ai[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    Ai[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (*sh)[kVecThreads], double* v,
                                                   double* part, int ti)
{
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kVecThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) part[NV * ti + k] = sh[k][0];
}

template <typename VT>
__global__ void __launch_bounds__(kVecThreads)
k_pcg_setup(const SceneDev* scenes, const Tile* tiles, int ntiles, double* part)
{
    __shared__ double sh[2][kVecThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    double v[2] = {0.0, 0.0};
    if (scene_live(S) && (int)threadIdx.x < T.count) {
        const int64_t n = T.start + threadIdx.x;
        double Mi[9];
        double b[3];
        if (S.pinned[n]) {
#pragma unroll
            for (int k = 0; k < 9; ++k) Mi[k] = (k % 4 == 0) ? 1.0 : 0.0;
            b[0] = b[1] = b[2] = 0.0;
        } else {
            const VT* vals = (sizeof(VT) == 8) ? (const VT*)S.vals64 : (const VT*)S.vals32;
            inv3x3<VT>(vals + 9 * (int64_t)S.diag_slot[n], Mi);
#pragma unroll
            for (int i = 0; i < 3; ++i) b[i] = -S.grad[3 * n + i];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) S.Minv[9 * n + k] = Mi[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double z = Mi[3 * i] * b[0] + Mi[3 * i + 1] * b[1] + Mi[3 * i + 2] * b[2];
            S.r[3 * n + i] = b[i];
            S.z[3 * n + i] = z;
            S.dx[3 * n + i] = 0.0;
            S.p0[3 * n + i] = 0.0;
            S.p1[3 * n + i] = 0.0;
            v[0] += b[i] * b[i];
            v[1] += b[i] * z;
        }
    }
    block_reduce_store<2>(sh, v, part, ti);
}

cudaError_t launch_pcg_setup_p(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                               int precision, double* part, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    if (precision == SX_FP32)
        k_pcg_setup<float><<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, part);
    else
        k_pcg_setup<double><<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ SpMV
// q = A p_new with p_new = z + beta p_old formed on the fly; one thread
// per block row. FP32 form: values and products in float, accumulation of
// each row in float, p cast to float on load.
template <typename VT>
__global__ void __launch_bounds__(kVecThreads)
k_spmv(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part)
{
    __shared__ double sh[1][kVecThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    double v[1] = {0.0};
    if (scene_live(S) && !S.sc->pcg_done && (int)threadIdx.x < T.count) {
        const int64_t r = T.start + threadIdx.x;
        const double beta = S.sc->pcg_beta;
        const double* po = par ? S.p1 : S.p0;
        double* pn = par ? S.p0 : S.p1;
        double pr[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pr[i] = S.z[3 * r + i] + beta * po[3 * r + i];
            pn[3 * r + i] = pr[i];
        }
        double q[3];
        if (S.pinned[r]) {
            q[0] = pr[0]; q[1] = pr[1]; q[2] = pr[2];
        } else {
            const VT* vals = (sizeof(VT) == 8) ? (const VT*)S.vals64 : (const VT*)S.vals32;
            VT acc[3] = {VT(0), VT(0), VT(0)};
            const int b = S.row_ptr[r], e = S.row_ptr[r + 1];
            for (int k = b; k < e; ++k) {
                const int c = S.col[k];
                if (S.pinned[c]) continue;
                VT pc[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) pc[j] = (VT)(S.z[3 * (int64_t)c + j] + beta * po[3 * (int64_t)c + j]);
                const VT* B = vals + 9 * (int64_t)k;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    acc[i] += B[3 * i] * pc[0] + B[3 * i + 1] * pc[1] + B[3 * i + 2] * pc[2];
            }
            q[0] = (double)acc[0]; q[1] = (double)acc[1]; q[2] = (double)acc[2];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S.q[3 * r + i] = q[i];
            v[0] += pr[i] * q[i];
        }
    }
    block_reduce_store<1>(sh, v, part, ti);
}

cudaError_t launch_spmv_pq(const SceneDev* scenes, const Tile* row_tiles, int ntiles,
                           int precision, int parity, double* part, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    if (precision == SX_FP32)
        k_spmv<float><<<ntiles, kVecThreads, 0, s>>>(scenes, row_tiles, ntiles, parity, part);
    else
        k_spmv<double><<<ntiles, kVecThreads, 0, s>>>(scenes, row_tiles, ntiles, parity, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ update
__global__ void __launch_bounds__(kVecThreads)
k_pcg_update(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part)
{
    __shared__ double sh[2][kVecThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    double v[2] = {0.0, 0.0};
    if (scene_live(S) && !S.sc->pcg_done && (int)threadIdx.x < T.count) {
        const int64_t n = T.start + threadIdx.x;
        const double alpha = S.sc->pcg_alpha;
        const double* pn = par ? S.p0 : S.p1;
        double r[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S.dx[3 * n + i] += alpha * pn[3 * n + i];
            r[i] = S.r[3 * n + i] - alpha * S.q[3 * n + i];
            S.r[3 * n + i] = r[i];
        }
        const double* Mi = S.Minv + 9 * n;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double z = Mi[3 * i] * r[0] + Mi[3 * i + 1] * r[1] + Mi[3 * i + 2] * r[2];
            S.z[3 * n + i] = z;
            v[0] += r[i] * z;
            v[1] += r[i] * r[i];
        }
    }
    block_reduce_store<2>(sh, v, part, ti);
}

cudaError_t launch_pcg_update(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                              int parity, double* part, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_pcg_update<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PCG scalars
// stage 0: after setup, part = [b.b, r.z] per node tile
// stage 1: after SpMV, part = [p.q] per row tile           -> alpha
// stage 2: after update, part = [r.z, r.r] per node tile    -> convergence, beta
__global__ void k_pcg_reduce(const double* part, int nv, const int* tbeg, const int* tend,
                             const SceneDev* scenes, int stage, double tol, int max_iter)
{
    __shared__ double sh[2][kRedT];
    const int s = blockIdx.x;
    SceneScal* sc = scenes[s].sc;
    if (!sc->active) return;
    if (stage > 0 && sc->pcg_done) return;
    double a = 0.0, b = 0.0;
    for (int t = tbeg[s] + threadIdx.x; t < tend[s]; t += kRedT) {
        a += part[(int64_t)t * nv];
        if (nv > 1) b += part[(int64_t)t * nv + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = kRedT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    a = sh[0][0];
    b = sh[1][0];
    if (stage == 0) {
        sc->bnorm2 = a;
        sc->rz = b;
        sc->rr = a;
        sc->pcg_iters = 0;
        sc->pcg_beta = 0.0;
        sc->pcg_status = 0;
        sc->pcg_done = (a == 0.0) ? 1 : 0;
    } else if (stage == 1) {
        sc->pq = a;
        if (!(a > 0.0) || !isfinite(a)) {   // not a descent system: stop
            sc->pcg_done = 1;
            sc->pcg_status = 1;
            sc->pcg_alpha = 0.0;
        } else {
            sc->pcg_alpha = sc->rz / a;
        }
    } else {
        sc->rz_new = a;
        sc->rr = b;
        sc->pcg_iters += 1;
        const double t = sc->pcg_tol > 0.0 ? sc->pcg_tol : tol;
        if (b <= t * t * sc->bnorm2) {
            sc->pcg_done = 1;
        } else if (sc->pcg_iters >= max_iter || !isfinite(b)) {
            sc->pcg_done = 1;
            sc->pcg_status = 2;
        } else {
            sc->pcg_beta = a / sc->rz;
            sc->rz = a;
        }
    }
}

cudaError_t launch_pcg_reduce(const double* part, int nv, const int* tbeg, const int* tend,
                              int nscenes, const SceneDev* scenes, int stage, double tol,
                              int max_iter, cudaStream_t s)
{
    if (!nscenes) return cudaSuccess;
    k_pcg_reduce<<<nscenes, kRedT, 0, s>>>(part, nv, tbeg, tend, scenes, stage, tol, max_iter);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ line search
// part per node tile: [g.dx]
__global__ void k_gdx(const SceneDev* scenes, const Tile* tiles, int ntiles, double* part)
{
    __shared__ double sh[1][kVecThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    double v[1] = {0.0};
    if (scene_live(S) && (int)threadIdx.x < T.count) {
        const int64_t n = T.start + threadIdx.x;
#pragma unroll
        for (int i = 0; i < 3; ++i) v[0] += S.grad[3 * n + i] * S.dx[3 * n + i];
    }
    block_reduce_store<1>(sh, v, part, ti);
}

cudaError_t launch_gdx(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                       double* part, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_gdx<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, part);
    return cudaGetLastError();
}

__global__ void k_trial(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || (int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
    const double a = S.sc->ls_alpha;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.x_trial[3 * n + i] = S.x[3 * n + i] + a * S.dx[3 * n + i];
}

cudaError_t launch_trial(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                         cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_trial<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles);
    return cudaGetLastError();
}

__global__ void k_accept(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || (int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.x[3 * n + i] = S.x_trial[3 * n + i];
}

cudaError_t launch_accept(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                          cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_accept<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles);
    return cudaGetLastError();
}

__global__ void k_velocity(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || (int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
    const double idt = 1.0 / S.dt;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.v[3 * n + i] = (S.x[3 * n + i] - S.x_start[3 * n + i]) * idt;
}

cudaError_t launch_velocity(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                            cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_velocity<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles);
    return cudaGetLastError();
}

}  // namespace sx
