// sx_solve.cu -- the backward-Euler Newton step's vector kernels (§3,
// Eqs. 2-3) and the 3x3 block-Jacobi preconditioned CG of §7.2, batched
// over scenes with per-scene scalars on the device.
//
// PCG iteration (per scene, x0 = 0, b = -g on free DOFs, 0 on pinned):
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

// ------------------------------------------------------------------ SpMV
// p_new = z + beta p_old (own rows), then q = A p_new. The direction update
// runs as its own vector pass so that the SpMV gathers a single vector and
// spends exactly 9 multiply-adds per 3x3 block (on GB300 the FP64 SpMV is
// bound by the FP64 pipe before HBM: 9 FMA per 76-byte block).
template <bool F32>
__global__ void __launch_bounds__(kVecThreads)
k_pcg_pdir(const SceneDev* scenes, const Tile* tiles, int ntiles, int par)
{
    const Tile T = tiles[blockIdx.x];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || S.sc->pcg_done || (int)threadIdx.x >= T.count) return;
    const int64_t n = T.start + threadIdx.x;
    const double beta = S.sc->pcg_beta;
    const double* po = par ? S.p1 : S.p0;
    double* pn = par ? S.p0 : S.p1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double p = fma(beta, po[3 * n + i], S.z[3 * n + i]);
        pn[3 * n + i] = p;
        // the FP32 SpMV gathers this rounded copy (no conversion per block)
        if (F32) S.p32[3 * n + i] = (float)p;
    }
}

cudaError_t launch_pcg_pdir(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                            int precision, int parity, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    if (precision == SX_FP32)
        k_pcg_pdir<true><<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity);
    else
        k_pcg_pdir<false><<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity);
    return cudaGetLastError();
}

// --- TMA bulk copy (non-tensor form) helpers: global -> shared, completion
// tracked by an mbarrier transaction count
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

#ifndef SX_SPMV_STAGE
#define SX_SPMV_STAGE 1
#endif
// 32 rows: 96 threads, three full warps (48 rows left half a warp idle);
// measured on the 64^3 cube, FP64 SpMV per call 134 us at 32 rows against
// 146 (48), 154 (64) and 165 (16); FP32 within 2% across 32-64. A form
// without staging (a half-warp per block row reading its blocks straight
// from global memory) measured 268 us: each lane's nine loads are 72 B apart
// from its neighbours', many sectors per load instruction. Splitting each
// output component over two threads (interleaved blocks, more warps for the
// same staged tile) made the 64^3 Newton step slower (224 vs 206 ms).
#ifndef SX_SPMV_ROWS
#define SX_SPMV_ROWS 32
#endif
static constexpr int kSpmvRows = SX_SPMV_ROWS;        // block rows per tile
static constexpr int kSpmvThreads = 3 * kSpmvRows;    // one thread per output component
// bytes of staged column ids and values: up to ~20 blocks per row (values in
// the value type), 1 KB granules; rows with more fall back to direct loads
static constexpr int kSpmvSmemCols = ((kSpmvRows * 4 * 1024 / 48) + 1023) / 1024 * 1024;
template <typename VT>
__host__ __device__ constexpr int spmv_smem_vals()
{
    return ((kSpmvRows * (sizeof(VT) == 8 ? 56 : 28) * 1024 / 48) + 1023) / 1024 * 1024;
}
__device__ __forceinline__ double fma_vt(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_vt(float a, float b, float c) { return fmaf(a, b, c); }
static constexpr long kWaitLimit = 1L << 24;          // bounded mbarrier wait

template <typename VT>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part,
       const int* tbeg, const int* tend)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double sh[1][kSpmvThreads];
    __shared__ int s_mode;   // 1: staged in shared memory, 0: direct loads
    __shared__ long s_vofs, s_cofs;
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    const bool live = scene_live(S) && !S.sc->pcg_done;
    const VT* vals = (sizeof(VT) == 8) ? (const VT*)S.vals64 : (const VT*)S.vals32;
    const int64_t r0 = T.start, r1 = T.start + T.count;
    if (threadIdx.x == 0) {
        s_mode = 0;
        if (live) {
            const int64_t k0 = S.row_ptr[r0], k1 = S.row_ptr[r1];
            // 16-byte aligned windows containing the tile's value and column
            // segments (the allocations are padded for the rounded-up end)
            const long vb0 = (long)(k0 * 9 * (int64_t)sizeof(VT)) & ~15L;
            const long vb1 = ((long)(k1 * 9 * (int64_t)sizeof(VT)) + 15L) & ~15L;
            const long cb0 = (long)(k0 * 4) & ~15L;
            const long cb1 = ((long)(k1 * 4) + 15L) & ~15L;
            if (SX_SPMV_STAGE && vb1 - vb0 <= spmv_smem_vals<VT>() && cb1 - cb0 <= kSpmvSmemCols &&
                k1 > k0) {
                s_mode = 1;
                s_vofs = vb0;
                s_cofs = cb0;
                mbar_init(&bar, 1);
                mbar_expect_tx(&bar, (unsigned)((vb1 - vb0) + (cb1 - cb0)));
                bulk_g2s(smem, (const unsigned char*)vals + vb0, (unsigned)(vb1 - vb0), &bar);
                bulk_g2s(smem + spmv_smem_vals<VT>(), (const unsigned char*)S.col + cb0,
                         (unsigned)(cb1 - cb0), &bar);
            }
        }
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode == 1) {
        long it = 0;
        while (!mbar_try_wait(&bar, 0) && ++it < kWaitLimit) {
        }
        if (it >= kWaitLimit) {
            // the copy did not complete in time: report it through the
            // scene's PCG status (the scene's last tile then stops its PCG),
            // wait (bounded) once more so that no write lands after exit, and
            // count the tile with a zero partial
            if (threadIdx.x == 0) S.sc->pcg_status = 3;
            long it2 = 0;
            while (!mbar_try_wait(&bar, 0) && ++it2 < kWaitLimit) {
            }
            const double z[1] = {0.0};
            double tot[1];
            if (last_tile_sums<1, kSpmvThreads>(z, sh, part, ti, &S.sc->cnt_spmv, tbeg[T.scene],
                                                tend[T.scene], tot) &&
                threadIdx.x == 0) {
                S.sc->pcg_done = 1;
                S.sc->pcg_alpha = 0.0;
            }
            return;
        }
    }
    double v = 0.0;
    const int lr = threadIdx.x / 3, ci = threadIdx.x - 3 * lr;
    if (live && lr < T.count) {
        const int64_t r = r0 + lr;
        const double* pn = par ? S.p0 : S.p1;
        double q;
        if (S.pinned[r]) {
            q = pn[3 * r + ci];
        } else {
            VT acc = VT(0);
            const int b = S.row_ptr[r], e = S.row_ptr[r + 1];
            // the gathered direction: p itself (FP64) or its float copy (FP32)
            const VT* pg = (sizeof(VT) == 8) ? (const VT*)pn : (const VT*)S.p32;
            const VT* vs = mode ? (const VT*)(smem + ((long)b * 9 * (long)sizeof(VT) - s_vofs))
                                : vals + 9 * (int64_t)b;
            const int* cs = mode ? (const int*)(smem + spmv_smem_vals<VT>() + ((long)b * 4 - s_cofs))
                                 : S.col + b;
            // p is exactly zero on pinned DOFs (their r, z and p stay 0), so
            // pinned columns drop out without a test in the loop
#pragma unroll 4
            for (int k = 0; k < e - b; ++k) {
                const int c = cs[k];
                const VT* B = vs + 9 * k + 3 * ci;
                // a chain of three fused multiply-adds: the minimum FP64
                // instruction count per block row
                acc = fma_vt(B[0], pg[3 * (int64_t)c], acc);
                acc = fma_vt(B[1], pg[3 * (int64_t)c + 1], acc);
                acc = fma_vt(B[2], pg[3 * (int64_t)c + 2], acc);
            }
            q = (double)acc;
        }
        S.q[3 * r + ci] = q;
        v = pn[3 * r + ci] * q;
    }
    if (!live) return;   // every tile of the scene sees the same state
    const double vv[1] = {v};
    double pq[1];
    if (last_tile_sums<1, kSpmvThreads>(vv, sh, part, ti, &S.sc->cnt_spmv, tbeg[T.scene],
                                        tend[T.scene], pq) &&
        threadIdx.x == 0) {
        SceneScal* sc = S.sc;
        sc->pq = pq[0];
        if (sc->pcg_status == 3) {
            sc->pcg_done = 1;
            sc->pcg_alpha = 0.0;
        } else if (!(pq[0] > 0.0) || !isfinite(pq[0])) {   // not a descent system: stop
            sc->pcg_done = 1;
            sc->pcg_status = 1;
            sc->pcg_alpha = 0.0;
        } else {
            sc->pcg_alpha = sc->rz / pq[0];
        }
    }
}

int spmv_rows_per_tile() { return kSpmvRows; }

void prepare_spmv()
{
    // the shared-memory opt-in is per device; contexts on several host
    // threads may reach this concurrently (setting it twice is harmless)
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (!bit || !(attr_done.load(std::memory_order_acquire) & bit)) {
        cudaFuncSetAttribute(k_spmv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             spmv_smem_vals<float>() + kSpmvSmemCols);
        cudaFuncSetAttribute(k_spmv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             spmv_smem_vals<double>() + kSpmvSmemCols);
        attr_done.fetch_or(bit, std::memory_order_release);
    }
}

cudaError_t launch_spmv_pq(const SceneDev* scenes, const Tile* row_tiles, int ntiles,
                           int precision, int parity, double* part, const int* tbeg,
                           const int* tend, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    const int smem64 = spmv_smem_vals<double>() + kSpmvSmemCols;
    const int smem32 = spmv_smem_vals<float>() + kSpmvSmemCols;
    prepare_spmv();
    if (precision == SX_FP32)
        k_spmv<float><<<ntiles, kSpmvThreads, smem32, s>>>(scenes, row_tiles, ntiles, parity, part,
                                                           tbeg, tend);
    else
        k_spmv<double><<<ntiles, kSpmvThreads, smem64, s>>>(scenes, row_tiles, ntiles, parity,
                                                            part, tbeg, tend);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ update
__global__ void __launch_bounds__(kVecThreads)
k_pcg_update(const SceneDev* scenes, const Tile* tiles, int ntiles, int par, double* part,
             const int* tbeg, const int* tend, double tol, int max_iter)
{
    __shared__ double sh[2][kVecThreads];
    const int ti = blockIdx.x;
    const Tile T = tiles[ti];
    const SceneDev& S = scenes[T.scene];
    if (!scene_live(S) || S.sc->pcg_done) return;   // the same for every tile of the scene
    double v[2] = {0.0, 0.0};
    if ((int)threadIdx.x < T.count) {
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
    double rzr[2];
    if (last_tile_sums<2, kVecThreads>(v, sh, part, ti, &S.sc->cnt_update, tbeg[T.scene],
                                       tend[T.scene], rzr) &&
        threadIdx.x == 0) {
        // convergence test and beta (the update of the chunk's p.q stage)
        SceneScal* sc = S.sc;
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

cudaError_t launch_pcg_update(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                              int parity, double* part, const int* tbeg, const int* tend,
                              double tol, int max_iter, cudaStream_t s)
{
    if (!ntiles) return cudaSuccess;
    k_pcg_update<<<ntiles, kVecThreads, 0, s>>>(scenes, node_tiles, ntiles, parity, part, tbeg,
                                                tend, tol, max_iter);
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
        cudaError_t e = cudaGraphAddKernelNode(&n, g, last ? &last : nullptr, last ? 1 : 0, &p);
        if (e == cudaSuccess) last = n;
        return e;
    }
};
}  // namespace

cudaError_t add_pcg_chunk_nodes(cudaGraph_t graph, const PcgChunkArgs& a)
{
    prepare_spmv();
    NodeChain c{graph};
    const bool f32 = a.precision == SX_FP32;
    const void* pdir = f32 ? (const void*)k_pcg_pdir<true> : (const void*)k_pcg_pdir<false>;
    const void* spmv = f32 ? (const void*)k_spmv<float> : (const void*)k_spmv<double>;
    const unsigned smem = (unsigned)(kSpmvSmemCols + (f32 ? spmv_smem_vals<float>()
                                                          : spmv_smem_vals<double>()));
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
        if (e == cudaSuccess) e = c.add(pdir, (unsigned)nnt, kVecThreads, 0, a_pdir);
        if (e == cudaSuccess) e = c.add(spmv, (unsigned)nrt, spmv_threads, smem, a_spmv);
        if (e == cudaSuccess) e = c.add((const void*)k_pcg_update, (unsigned)nnt, kVecThreads, 0, a_upd);
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
