// sx_solve.cu -- the backward-Euler Newton step's vector kernels (§3,
// Eqs. 2-3) and the 3x3 block-Jacobi preconditioned CG of §7.2, batched
// over scenes with per-scene scalars on the device.
//
// The setup also copies the assembled values into the SpMV's sliced
// layout (below). PCG iteration (per scene, x0 = 0, b = -g on free DOFs, 0
// on pinned):
//   p_new = z + beta p_old;  q = A p_new;  alpha = (r.z) / (p_new.q)
//   dx += alpha p_new;  r -= alpha q;  z = Minv r
//   stop when ||r|| <= tol ||b||;  beta = r.z_new / r.z
// p_old and p_new alternate between two buffers. An iteration is three
// kernels: direction; SpMV with the p.q partials, whose last tile per scene
// sums them and forms alpha; update with the r.z and r.r partials, whose
// last tile per scene sums them, tests convergence and forms beta. Pinned
// DOFs are eliminated by mask: their rows are identity, and their columns
// drop out because p is zero there.
#include <cuda_runtime.h>

#include <atomic>

#include <cuda/atomic>

#include "sx_internal.cuh"

namespace sx {

static constexpr int kVecThreads = 256;
static constexpr int kRedT = 256;

__device__ __forceinline__ bool scene_live(const SceneDev& S)
{
    return S.sc == nullptr || S.sc->active;
}

// In the PCG chunk graph each iteration kernel may be launched before the
// one it depends on has finished (a programmatic edge from that kernel's
// launch completion); it waits here, before reading anything the previous
// kernel writes, until that kernel has completed and its writes are
// visible. Without such an edge (plain launches) this returns at once.
#ifndef SX_PCG_PDL
#define SX_PCG_PDL 1
#endif
__device__ __forceinline__ void wait_prior_grid()
{
#if SX_PCG_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
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
        // this row into the SpMV's sliced copy (node tiles start at multiples
        // of 256, so the 32 lanes of a warp fill one slice: coalesced stores)
        {
            const VT* vals = (sizeof(VT) == 8) ? (const VT*)S.vals64 : (const VT*)S.vals32;
            VT* sv = (sizeof(VT) == 8) ? (VT*)S.sell_v64 : (VT*)S.sell_v32;
            const int64_t sl = n >> 5;
            const int k0 = S.sell_ptr[sl], w = S.sell_ptr[sl + 1] - k0;
            const int b = S.row_ptr[n], len = S.pinned[n] ? 0 : S.row_ptr[n + 1] - b;
            VT* dst = sv + (int64_t)k0 * 288 + (n & 31);
            const VT* src = vals + 9 * (int64_t)b;
            for (int k = 0; k < w; ++k)
#pragma unroll
                for (int e = 0; e < 9; ++e)
                    __stcs(dst + (int64_t)288 * k + 32 * e, k < len ? src[9 * k + e] : VT(0));
        }
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

// ------------------------------------------------------------------ scene sums in the last tile
// Each tile of a live scene stores its partial(s), then counts itself done
// on the scene's counter; the block that completes the count sums the
// scene's partials over its tile range in a fixed order (so the result does
// not depend on which block was last) and resets the counter.
template <int NV, int NT>
__device__ __forceinline__ bool last_tile_sums(const double (&v)[NV], double (*sh)[NT],
                                               double* part, int ti, int* counter, int tb,
                                               int te, double (&out)[NV])
{
    __shared__ int s_last;
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w && (int)threadIdx.x + w < NT)
#pragma unroll
            for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(int64_t)NV * ti + k] = sh[k][0];
        // release: this tile's partial is visible to whoever counts last;
        // acquire: the last one sees every partial released before it
        cuda::atomic_ref<int, cuda::thread_scope_device> cnt(*counter);
        s_last = cnt.fetch_add(1, cuda::memory_order_acq_rel) == te - tb - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    // four interleaved accumulators per thread (independent loads and adds),
    // combined in a fixed order
    double a[4][NV];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < NV; ++k) a[j][k] = 0.0;
    int t = tb + threadIdx.x;
    for (; t + 3 * NT < te; t += 4 * NT)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < NV; ++k) a[j][k] += __ldcg(part + (int64_t)NV * (t + j * NT) + k);
#pragma unroll
    for (int j = 0; j < 3; ++j)   // fewer than 4 strides left
        if (t < te) {
#pragma unroll
            for (int k = 0; k < NV; ++k) a[j][k] += __ldcg(part + (int64_t)NV * t + k);
            t += NT;
        }
#pragma unroll
    for (int k = 0; k < NV; ++k) a[0][k] = (a[0][k] + a[1][k]) + (a[2][k] + a[3][k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = a[0][k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w && (int)threadIdx.x + w < NT)
#pragma unroll
            for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = sh[k][0];
    if (threadIdx.x == 0) *counter = 0;
    return true;
}

// The pieces of last_tile_sums for blocks that handle several tiles: the
// sum of a scene's NV-value tile partials over its tile range [tb, te) in a
// fixed order (every thread of the block takes part; the result on all).
template <int NV, int NT>
__device__ __forceinline__ void scene_tile_sums(double (*sh)[NT], const double* part, int tb,
                                                int te, double (&out)[NV])
{
    double a[4][NV];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < NV; ++k) a[j][k] = 0.0;
    int t = tb + threadIdx.x;
    for (; t + 3 * NT < te; t += 4 * NT)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < NV; ++k) a[j][k] += __ldcg(part + (int64_t)NV * (t + j * NT) + k);
#pragma unroll
    for (int j = 0; j < 3; ++j)   // fewer than 4 strides left
        if (t < te) {
#pragma unroll
            for (int k = 0; k < NV; ++k) a[j][k] += __ldcg(part + (int64_t)NV * t + k);
            t += NT;
        }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = (a[0][k] + a[1][k]) + (a[2][k] + a[3][k]);
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w && (int)threadIdx.x + w < NT)
#pragma unroll
            for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = sh[k][0];
    __syncthreads();
}

// ------------------------------------------------------------------ SpMV
// p_new = z + beta p_old (own rows), then q = A p_new. The direction update
// runs as its own vector pass so that the SpMV gathers a single vector and
// spends exactly 9 multiply-adds per 3x3 block (on GB300 the FP64 SpMV is
// bound by the FP64 pipe before HBM: 9 FMA per 76-byte block).
#ifndef SX_UPD_TILES
#define SX_UPD_TILES 1
#endif
static constexpr int kUpdTiles = SX_UPD_TILES;
int pcg_update_blocks(int n_node_tiles) { return (n_node_tiles + kUpdTiles - 1) / kUpdTiles; }

// The update (below) with half the threads: a 128-thread block per 256-node
// tile, thread t taking nodes t and t + 128 (loads of both first). Each
// thread adds its two nodes' r.z and r.r in node order; lane l of warp 0
// then adds the partials of threads l, l + 32, l + 64, l + 96 in that order
// and the warp finishes with a fixed shuffle tree, so a tile's partial (and
// the scene sums, folded by the last tile as above) depends only on the
// tile's data. On this GPU the update is bound by the FP64 pipe, which a
// 256-thread shared-memory tree with nine barriers per tile kept waiting.
#ifndef SX_UPD_SPLIT
#define SX_UPD_SPLIT 1
#endif
constexpr int kUpd2Threads = 128;
// resident blocks per SM the two-node update is compiled for (a register
// cap; 0: none, 106 registers, four blocks). Caps for 5, 6 and 8 blocks (96,
// 80, 64 registers, with spills) measured no faster on the 64^3 cube's
// Newton step: 113.0, 112.5, 111.3 against 111.1 ms
#ifndef SX_UPD2_MINB
#define SX_UPD2_MINB 0
#endif

__device__ __forceinline__ double warp_sum_xor(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kUpd2Threads, SX_UPD2_MINB > 0 ? SX_UPD2_MINB : 1)
k_pcg_update2(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part,
              const int* tbeg, const int* tend, double tol, int max_iter)
{
    wait_prior_grid();
    __shared__ double sh[2][kUpd2Threads];
    __shared__ int s_last;
    const int ti = blockIdx.x;
    if (ti >= ntiles) return;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || S.sc->pcg_done) return;   // the same for all tiles of a scene
    const double alpha = S.sc->pcg_alpha;
    const double* pn = par ? S.p0 : S.p1;
    double pv[2][3], dxv[2][3], rv[2][3], qv[2][3], Mi[2][9];
    bool on[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int l = (int)threadIdx.x + kUpd2Threads * h;
        on[h] = l < T.count;
        if (!on[h]) continue;
        const int64_t n = T.start + l;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pv[h][i] = pn[3 * n + i];
            dxv[h][i] = S.dx[3 * n + i];
            rv[h][i] = S.r[3 * n + i];
            qv[h][i] = S.q[3 * n + i];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) Mi[h][k] = S.Minv[9 * n + k];
    }
    double rz = 0.0, rr = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!on[h]) continue;
        const int64_t n = T.start + (int)threadIdx.x + kUpd2Threads * h;
        double r[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S.dx[3 * n + i] = dxv[h][i] + alpha * pv[h][i];
            r[i] = rv[h][i] - alpha * qv[h][i];
            S.r[3 * n + i] = r[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double z = Mi[h][3 * i] * r[0] + Mi[h][3 * i + 1] * r[1] + Mi[h][3 * i + 2] * r[2];
            S.z[3 * n + i] = z;
            rz += r[i] * z;
            rr += r[i] * r[i];
        }
    }
    sh[0][threadIdx.x] = rz;
    sh[1][threadIdx.x] = rr;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        double a = ((sh[0][l] + sh[0][l + 32]) + sh[0][l + 64]) + sh[0][l + 96];
        double b = ((sh[1][l] + sh[1][l + 32]) + sh[1][l + 64]) + sh[1][l + 96];
        a = warp_sum_xor(a);
        b = warp_sum_xor(b);
        if (l == 0) {
            part[2 * (int64_t)ti] = a;
            part[2 * (int64_t)ti + 1] = b;
            // release: this tile's partials are visible to whoever counts
            // last; acquire: the last one sees every partial released before it
            cuda::atomic_ref<int, cuda::thread_scope_device> cnt(S.sc->cnt_update);
            s_last = cnt.fetch_add(1, cuda::memory_order_acq_rel) == tend[T.scene] - tbeg[T.scene] - 1;
        }
    }
    __syncthreads();
    if (!s_last) return;
    double rzr[2];
    scene_tile_sums<2, kUpd2Threads>(sh, part, tbeg[T.scene], tend[T.scene], rzr);
    if (threadIdx.x == 0) {
        // convergence test and beta
        SceneScal* sc = S.sc;
        sc->cnt_update = 0;
        sc->rz_new = rzr[0];
        sc->rr = rzr[1];
        sc->pcg_iters += 1;
        const double t = sc->pcg_tol > 0.0 ? sc->pcg_tol : tol;
        if (rzr[1] <= t * t * sc->bnorm2) {
            sc->pcg_done = 1;
        } else if (sc->pcg_iters >= max_iter || !isfinite(rzr[1])) {
            sc->pcg_done = 1;
            sc->pcg_status = 2;
        } else {
            sc->pcg_beta = rzr[0] / sc->rz;
            sc->rz = rzr[0];
        }
    }
}

// the direction pass with the same thread layout (two nodes per thread)
template <bool F32>
__global__ void __launch_bounds__(kUpd2Threads)
k_pcg_pdir2(const SceneDev* scenes, const Tile* tiles, int ntiles, int par)
{
    wait_prior_grid();
    const int ti = blockIdx.x;
    if (ti >= ntiles) return;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || S.sc->pcg_done) return;
    const double beta = S.sc->pcg_beta;
    const double* po = par ? S.p1 : S.p0;
    double* pw = par ? S.p0 : S.p1;
    double zv[2][3], ov[2][3];
    bool on[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int l = (int)threadIdx.x + kUpd2Threads * h;
        on[h] = l < T.count;
        if (!on[h]) continue;
        const int64_t n = T.start + l;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ov[h][i] = po[3 * n + i];
            zv[h][i] = S.z[3 * n + i];
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!on[h]) continue;
        const int64_t n = T.start + (int)threadIdx.x + kUpd2Threads * h;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double p = fma(beta, ov[h][i], zv[h][i]);
            pw[3 * n + i] = p;
            // the FP32 SpMV gathers this rounded copy (no conversion per block)
            if (F32) S.p32[3 * n + i] = (float)p;
        }
    }
}

template <bool F32>
__global__ void __launch_bounds__(kVecThreads)
k_pcg_pdir(const SceneDev* scenes, const Tile* tiles, int ntiles, int par)
{
    wait_prior_grid();
    // kUpdTiles node tiles per block, loads first (as in the update)
    double zv[kUpdTiles][3], ov[kUpdTiles][3], beta[kUpdTiles];
    bool on[kUpdTiles];
    int64_t nd[kUpdTiles];
    const int t0 = blockIdx.x * kUpdTiles;
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        on[j] = false;
        if (t0 + j >= ntiles) continue;
        const Tile T = tiles[t0 + j];
        const SceneDev& S = scenes[T.scene];
        on[j] = scene_live(S) && !S.sc->pcg_done && (int)threadIdx.x < T.count;
        if (!on[j]) continue;
        const int64_t n = T.start + threadIdx.x;
        nd[j] = n;
        beta[j] = S.sc->pcg_beta;
        const double* po = par ? S.p1 : S.p0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ov[j][i] = po[3 * n + i];
            zv[j][i] = S.z[3 * n + i];
        }
    }
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        if (!on[j]) continue;
        const SceneDev& S = scenes[tiles[t0 + j].scene];
        const int64_t n = nd[j];
        double* pn = par ? S.p0 : S.p1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double p = fma(beta[j], ov[j][i], zv[j][i]);
            pn[3 * n + i] = p;
            // the FP32 SpMV gathers this rounded copy (no conversion per block)
            if (F32) S.p32[3 * n + i] = (float)p;
        }
    }
}

cudaError_t launch_pcg_pdir(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                            int precision, int parity, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    const int g = pcg_update_blocks(ntiles);
    if (SX_UPD_SPLIT) {
        if (precision == SX_FP32)
            k_pcg_pdir2<true><<<ntiles, kUpd2Threads, 0, s>>>(scenes, node_tiles, ntiles, parity);
        else
            k_pcg_pdir2<false><<<ntiles, kUpd2Threads, 0, s>>>(scenes, node_tiles, ntiles, parity);
    } else if (precision == SX_FP32) {
        k_pcg_pdir<true><<<g, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity);
    } else {
        k_pcg_pdir<false><<<g, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ SpMV layout
// The PCG multiplies with a copy of the BSR values in sliced-ELLPACK form.
// A slice is 32 consecutive block rows (one warp, one lane per block row),
// padded to its longest row; entry (slice s, step k, lane l) is the k-th
// block of row 32 s + l. The blocks are stored [step][9 entries][32 lanes],
// so each of a warp's value loads is one contiguous segment (256 bytes in
// FP64, 128 in FP32) and the matrix streams from HBM with no staging and no
// idle lanes. sell_ptr[s] counts the steps of the slices before s. Pad
// entries hold zeros and a valid column (the row's own). The columns are
// laid out once per pattern; the values are copied from the BSR in the PCG
// setup, with pinned rows as zeros (their q = A p is then 0, which equals p
// there: p stays zero on pinned DOFs).
__global__ void k_sell_widths(const int* __restrict__ row_ptr, int64_t N, int* __restrict__ w)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= (N + 31) / 32) return;
    int m = 0;
    const int64_t r1 = min(N, 32 * s + 32);
    for (int64_t r = 32 * s; r < r1; ++r) m = max(m, row_ptr[r + 1] - row_ptr[r]);
    w[s] = m;
}

__global__ void k_sell_cols(const int* __restrict__ row_ptr, const int* __restrict__ col,
                            int64_t N, const int* __restrict__ sell_ptr, int* __restrict__ sell_col)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // 32 s + lane
    if (r >= 32 * ((N + 31) / 32)) return;
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const int k0 = sell_ptr[s], w = sell_ptr[s + 1] - k0;
    const bool real = r < N;
    const int b = real ? row_ptr[r] : 0, len = real ? row_ptr[r + 1] - b : 0;
    const int own = real ? (int)r : (int)(32 * s);
    for (int k = 0; k < w; ++k)
        sell_col[((int64_t)(k0 + k) << 5) + lane] = k < len ? col[b + k] : own;
}

cudaError_t launch_sell_widths(const int* row_ptr, int64_t N, int* widths, cudaStream_t s)
{
    const int64_t nsl = (N + 31) / 32;
    if (!nsl) return cudaSuccess;
    k_sell_widths<<<(unsigned)((nsl + 255) / 256), 256, 0, s>>>(row_ptr, N, widths);
    return cudaGetLastError();
}

cudaError_t launch_sell_cols(const int* row_ptr, const int* col, int64_t N, const int* sell_ptr,
                             int* sell_col, cudaStream_t s)
{
    const int64_t nr = 32 * ((N + 31) / 32);
    if (!nr) return cudaSuccess;
    k_sell_cols<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(row_ptr, col, N, sell_ptr, sell_col);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ SpMV
// q = A p_new over the sliced copy of A, with the p.q partials. A tile is
// four slices (128 block rows, four warps); lane l of warp w takes block
// row start + 32 w + l and its three output components, as three chains of
// fused multiply-adds over the row's blocks in column order (on GB300 the
// FP64 SpMV is bound by the FP64 pipe before HBM: 9 FMA per 76-byte block,
// the minimum). The matrix is read once, with evict-first loads so that the
// gathered direction (L2-resident, ~7 MB per million rows) stays cached.
#ifndef SX_SPMV_SLICES
#define SX_SPMV_SLICES 4
#endif
#ifndef SX_SPMV_UNROLL
#define SX_SPMV_UNROLL 2
#endif
static constexpr int kSpmvSlices = SX_SPMV_SLICES;
static constexpr int kSpmvUnroll = SX_SPMV_UNROLL;
static constexpr int kSpmvRows = 32 * kSpmvSlices;   // block rows per tile
static constexpr int kSpmvThreads = kSpmvRows;       // one thread per block row
__device__ __forceinline__ double fma_vt(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_vt(float a, float b, float c) { return fmaf(a, b, c); }

template <typename VT>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part,
       const int* tbeg, const int* tend)
{
    wait_prior_grid();
    __shared__ double sh[1][kSpmvThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || S.sc->pcg_done) return;   // the same for every tile of the scene
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* pn = par ? S.p0 : S.p1;
    double v = 0.0;
    if (32 * warp < T.count) {
        // tiles start at multiples of 128 rows: warp w owns slice start/32 + w
        const int64_t sl = (T.start >> 5) + warp;
        const int k0 = S.sell_ptr[sl], w = S.sell_ptr[sl + 1] - k0;
        const VT* vs = (sizeof(VT) == 8 ? (const VT*)S.sell_v64 : (const VT*)S.sell_v32) +
                       (int64_t)k0 * 288 + lane;
        const int* cs = S.sell_col + ((int64_t)k0 << 5) + lane;
        // the gathered direction: p itself (FP64) or its float copy (FP32)
        const VT* pg = (sizeof(VT) == 8) ? (const VT*)pn : (const VT*)S.p32;
        VT a0 = VT(0), a1 = VT(0), a2 = VT(0);
#pragma unroll kSpmvUnroll
        for (int k = 0; k < w; ++k) {
            const int64_t c = 3 * (int64_t)__ldcs(cs + 32 * k);
            const VT x0 = __ldg(pg + c), x1 = __ldg(pg + c + 1), x2 = __ldg(pg + c + 2);
            const VT* B = vs + (int64_t)288 * k;
            a0 = fma_vt(__ldcs(B), x0, a0);
            a0 = fma_vt(__ldcs(B + 32), x1, a0);
            a0 = fma_vt(__ldcs(B + 64), x2, a0);
            a1 = fma_vt(__ldcs(B + 96), x0, a1);
            a1 = fma_vt(__ldcs(B + 128), x1, a1);
            a1 = fma_vt(__ldcs(B + 160), x2, a1);
            a2 = fma_vt(__ldcs(B + 192), x0, a2);
            a2 = fma_vt(__ldcs(B + 224), x1, a2);
            a2 = fma_vt(__ldcs(B + 256), x2, a2);
        }
        if ((int)threadIdx.x < T.count) {
            const int64_t r = T.start + threadIdx.x;
            const double q0 = (double)a0, q1 = (double)a1, q2 = (double)a2;
            S.q[3 * r] = q0;
            S.q[3 * r + 1] = q1;
            S.q[3 * r + 2] = q2;
            v = pn[3 * r] * q0 + pn[3 * r + 1] * q1 + pn[3 * r + 2] * q2;
        }
    }
    const double vv[1] = {v};
    double pq[1];
    if (last_tile_sums<1, kSpmvThreads>(vv, sh, part, ti, &S.sc->cnt_spmv, tbeg[T.scene],
                                        tend[T.scene], pq) &&
        threadIdx.x == 0) {
        SceneScal* sc = S.sc;
        sc->pq = pq[0];
        if (!(pq[0] > 0.0) || !isfinite(pq[0])) {   // not a descent system: stop
            sc->pcg_done = 1;
            sc->pcg_status = 1;
            sc->pcg_alpha = 0.0;
        } else {
            sc->pcg_alpha = sc->rz / pq[0];
        }
    }
}

int spmv_rows_per_tile() { return kSpmvRows; }

cudaError_t launch_spmv_pq(const SceneDev* scenes, const Tile* row_tiles, int ntiles,
                           int precision, int parity, double* part, const int* tbeg,
                           const int* tend, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    if (precision == SX_FP32)
        k_spmv<float><<<ntiles, kSpmvThreads, 0, s>>>(scenes, row_tiles, ntiles, parity, part,
                                                      tbeg, tend);
    else
        k_spmv<double><<<ntiles, kSpmvThreads, 0, s>>>(scenes, row_tiles, ntiles, parity, part,
                                                       tbeg, tend);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ update
// dx += alpha p, r -= alpha q, z = Minv r with the r.z and r.r partials per
// node tile; the last tile of each scene forms its convergence test and
// beta. A block takes kUpdTiles consecutive node tiles (a build parameter:
// their loads issued together, one block prologue for several tiles); each
// tile's partials are reduced by the same 256-thread tree as a block of its
// own, so the sums do not depend on how tiles are grouped. Measured on the
// 64^3 cube's Newton step: 1 and 2 tiles per block alike (153 ms), 4 slower
// (160 ms: the registers of four tiles halve the resident blocks); capping
// the registers for 7 or 8 resident blocks (one wave of the cube's 1,073
// tiles) changed nothing (154 ms).
__global__ void __launch_bounds__(kVecThreads)
k_pcg_update(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part,
             const int* tbeg, const int* tend, double tol, int max_iter)
{
    wait_prior_grid();
    __shared__ double sh[2 * kUpdTiles][kVecThreads];
    __shared__ int s_last[kUpdTiles];
    const int t0 = blockIdx.x * kUpdTiles;
    double rr_[kUpdTiles], rz_[kUpdTiles];
    bool live[kUpdTiles];
    double pv[kUpdTiles][3], dxv[kUpdTiles][3], rv[kUpdTiles][3], qv[kUpdTiles][3],
        Mi[kUpdTiles][9], alpha[kUpdTiles];
    int64_t nd[kUpdTiles];
    bool on[kUpdTiles];
    // loads of every tile first
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        live[j] = false;
        on[j] = false;
        const int ti = t0 + j;
        if (ti >= ntiles) continue;
        const Tile T = tiles[ti];
        const SceneDev& S = scenes[T.scene];
        live[j] = scene_live(S) && !S.sc->pcg_done;   // the same for all tiles of a scene
        on[j] = live[j] && (int)threadIdx.x < T.count;
        if (!on[j]) continue;
        const int64_t n = T.start + threadIdx.x;
        nd[j] = n;
        alpha[j] = S.sc->pcg_alpha;
        const double* pn = par ? S.p0 : S.p1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pv[j][i] = pn[3 * n + i];
            dxv[j][i] = S.dx[3 * n + i];
            rv[j][i] = S.r[3 * n + i];
            qv[j][i] = S.q[3 * n + i];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) Mi[j][k] = S.Minv[9 * n + k];
    }
    // arithmetic and stores
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        rz_[j] = 0.0;
        rr_[j] = 0.0;
        if (!on[j]) continue;
        const SceneDev& S = scenes[tiles[t0 + j].scene];
        const int64_t n = nd[j];
        double r[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            S.dx[3 * n + i] = dxv[j][i] + alpha[j] * pv[j][i];
            r[i] = rv[j][i] - alpha[j] * qv[j][i];
            S.r[3 * n + i] = r[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double z = Mi[j][3 * i] * r[0] + Mi[j][3 * i + 1] * r[1] + Mi[j][3 * i + 2] * r[2];
            S.z[3 * n + i] = z;
            rz_[j] += r[i] * z;
            rr_[j] += r[i] * r[i];
        }
    }
    // per tile: the 256-thread tree, the partials, the count
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        sh[2 * j][threadIdx.x] = rz_[j];
        sh[2 * j + 1][threadIdx.x] = rr_[j];
    }
    __syncthreads();
    for (int w = kVecThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 2 * kUpdTiles; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < kUpdTiles; ++j) {
            s_last[j] = 0;
            if (!live[j]) continue;
            const int ti = t0 + j;
            const Tile T = tiles[ti];
            const SceneDev& S = scenes[T.scene];
            part[2 * (int64_t)ti] = sh[2 * j][0];
            part[2 * (int64_t)ti + 1] = sh[2 * j + 1][0];
            // release: this tile's partials are visible to whoever counts
            // last; acquire: the last one sees every partial released before it
            cuda::atomic_ref<int, cuda::thread_scope_device> cnt(S.sc->cnt_update);
            s_last[j] = cnt.fetch_add(1, cuda::memory_order_acq_rel) ==
                        tend[T.scene] - tbeg[T.scene] - 1;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kUpdTiles; ++j) {
        if (!s_last[j]) continue;
        const int sc_i = tiles[t0 + j].scene;
        double rzr[2];
        scene_tile_sums<2, kVecThreads>(sh, part, tbeg[sc_i], tend[sc_i], rzr);
        if (threadIdx.x == 0) {
            // convergence test and beta
            SceneScal* sc = scenes[sc_i].sc;
            sc->cnt_update = 0;
            sc->rz_new = rzr[0];
            sc->rr = rzr[1];
            sc->pcg_iters += 1;
            const double t = sc->pcg_tol > 0.0 ? sc->pcg_tol : tol;
            if (rzr[1] <= t * t * sc->bnorm2) {
                sc->pcg_done = 1;
            } else if (sc->pcg_iters >= max_iter || !isfinite(rzr[1])) {
                sc->pcg_done = 1;
                sc->pcg_status = 2;
            } else {
                sc->pcg_beta = rzr[0] / sc->rz;
                sc->rz = rzr[0];
            }
        }
    }
}

cudaError_t launch_pcg_update(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                              int parity, double* part, const int* tbeg, const int* tend,
                              double tol, int max_iter, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    if (SX_UPD_SPLIT)
        k_pcg_update2<<<ntiles, kUpd2Threads, 0, s>>>(scenes, node_tiles, ntiles, parity, part,
                                                      tbeg, tend, tol, max_iter);
    else
        k_pcg_update<<<pcg_update_blocks(ntiles), kVecThreads, 0, s>>>(
            scenes, node_tiles, ntiles, parity, part, tbeg, tend, tol, max_iter);
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
        sc->cnt_spmv = 0;
        sc->cnt_update = 0;
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

// ------------------------------------------------------------------ PCG chunk graph
// The eight iterations of launch order (direction, SpMV with the p.q sums,
// update with the r.z / r.r sums) as kernel nodes of an explicitly built graph, each
// node depending on the one before: the same kernels, arguments and order as
// the plain launches. Built without stream capture, so host threads of other
// contexts may synchronize the device while it is built.
namespace {
struct NodeChain {
    cudaGraph_t g;
    cudaGraphNode_t last = nullptr;
    cudaError_t add(const void* func, unsigned grid, unsigned block, unsigned smem, void** args)
    {
        if (grid == 0) return cudaSuccess;
        cudaKernelNodeParams p{};
        p.func = const_cast<void*>(func);
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = smem;
        p.kernelParams = args;
        p.extra = nullptr;
        cudaGraphNode_t n = nullptr;
#if SX_PCG_PDL
        cudaError_t e = cudaGraphAddKernelNode(&n, g, nullptr, 0, &p);
        if (e == cudaSuccess && last) {
            // programmatic edge: the node may launch once every block of
            // `last` has started; it waits (wait_prior_grid) for its completion
            cudaGraphEdgeData ed{};
            ed.from_port = cudaGraphKernelNodePortLaunchCompletion;
            ed.to_port = 0;
            ed.type = cudaGraphDependencyTypeProgrammatic;
            e = cudaGraphAddDependencies(g, &last, &n, &ed, 1);
        }
#else
        cudaError_t e = cudaGraphAddKernelNode(&n, g, last ? &last : nullptr, last ? 1 : 0, &p);
#endif
        if (e == cudaSuccess) last = n;
        return e;
    }
};
}  // namespace

cudaError_t add_pcg_chunk_nodes(cudaGraph_t graph, const PcgChunkArgs& a)
{
    NodeChain c{graph};
    const bool f32 = a.precision == SX_FP32;
    const void* pdir = SX_UPD_SPLIT
                           ? (f32 ? (const void*)k_pcg_pdir2<true> : (const void*)k_pcg_pdir2<false>)
                           : (f32 ? (const void*)k_pcg_pdir<true> : (const void*)k_pcg_pdir<false>);
    const void* upd = SX_UPD_SPLIT ? (const void*)k_pcg_update2 : (const void*)k_pcg_update;
    const unsigned upd_grid = SX_UPD_SPLIT ? (unsigned)a.n_node_tiles
                                           : (unsigned)pcg_update_blocks(a.n_node_tiles);
    const unsigned upd_threads = SX_UPD_SPLIT ? kUpd2Threads : kVecThreads;
    const void* spmv = f32 ? (const void*)k_spmv<float> : (const void*)k_spmv<double>;
    const unsigned smem = 0;
    const unsigned spmv_threads = kSpmvThreads;
    // argument values must outlive each cudaGraphAddKernelNode call only
    const SceneDev* scenes = a.scenes;
    const Tile* nt = a.node_tiles;
    const Tile* rt = a.row_tiles;
    int nnt = a.n_node_tiles, nrt = a.n_row_tiles;
    double* prow = a.part_row;
    double* pnode = a.part_node;
    const int *rb = a.row_beg, *re = a.row_end, *nb = a.node_beg, *ne = a.node_end;
    double tol = a.tol;
    int maxit = a.max_iter;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < 8 && e == cudaSuccess; ++j) {
        int par = j & 1;
        void* a_pdir[] = {&scenes, &nt, &nnt, &par};
        void* a_spmv[] = {&scenes, &rt, &nrt, &par, &prow, &rb, &re};
        void* a_upd[] = {&scenes, &nt, &nnt, &par, &pnode, &nb, &ne, &tol, &maxit};
        if (e == cudaSuccess) e = c.add(pdir, upd_grid, upd_threads, 0, a_pdir);
        if (e == cudaSuccess) e = c.add(spmv, (unsigned)nrt, spmv_threads, smem, a_spmv);
        if (e == cudaSuccess) e = c.add(upd, upd_grid, upd_threads, 0, a_upd);
    }
    return e;
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

// a failed step is not taken: x back to the start of the step
__global__ void k_restore(const SceneDev* scenes, const Tile* tiles, int ntiles)
{
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || (int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.x[3 * n + i] = S.x_start[3 * n + i];
}

cudaError_t launch_restore(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                           cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_restore<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles);
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
