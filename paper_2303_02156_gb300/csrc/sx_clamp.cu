// sx_clamp.cu -- phase 2 of the per-element projection to positive
// semi-definiteness (§5.2 "Projection to positive semi-definiteness",
// Algorithm 1): the queued 9x9 translation-free Hessians are
// eigen-decomposed (float Jacobi; then, in double, a certified refinement of
// the subspace of the k <= 3 lowest eigenvalues, or Gram-Schmidt and
// block-restricted Jacobi sweeps for the other k: sx_clamp.cuh), their
// negative eigenvalues clamped and the stencils' Hessian blocks rewritten.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "sx_elements.cuh"

namespace sx {

// stencils with an N block of 1..3 columns: subspace refinement (1) or the
// block-restricted double Jacobi of every other k (0)
#ifndef SX_CLAMP_REFINE
#define SX_CLAMP_REFINE 1
#endif
// stencils of k >= 4 with 1..3 clearly negative modes: deflation of those
// (1) or the block-restricted double Jacobi (0)
#ifndef SX_CLAMP_DEFL
#define SX_CLAMP_DEFL 1
#endif

// After the eigen-decomposition: flags a non-finite result, else clamps
// the N-block eigenvalues below -tau in the Hadamard basis and rewrites the
// stencil's Hessian blocks (both projection launches end with this).
template <typename HT>
__device__ __forceinline__ void clamp_finish(const ElemLaunch& L, const ClampRef& ref,
                                             const double* __restrict__ Mg, const SmemMat& X,
                                             const double (&lam)[9], int k, double tau,
                                             unsigned live)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) ok = ok && isfinite(lam[i]);
    if (!ok) {
        atomicAdd(L.clamp_failed, 1);
        atomicExch(&L.scenes[ref.scene].sc->clamp_fail, 1);
        return;
    }
    const SceneDev& S = L.scenes[ref.scene];
    const ElemBlock& B = S.blk[ref.blk];
    HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * (B.base + ref.e);
    double* full = L.out_H ? L.out_H + 144 * ref.e : nullptr;
    // M' = M - sum of lambda v v^T over the N-block eigenvalues below -tau
    // (v in the Hadamard basis), then H' = (Hd kron I3) diag(0, M')
    // (Hd kron I3)^T written once: no read of the staged H, one store per
    // entry whatever the number of negative eigenvalues. (The element H
    // has the three translations as an exact null space up to rounding,
    // so H' differs from H - sum lambda u u^T only by rounding.)
    bool any_neg = false;
    double Mp[45];
#pragma unroll
    for (int q = 0; q < 45; ++q) Mp[q] = __ldg(Mg + q);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool neg = i < k && lam[i] < -tau;
        if (!__any_sync(live, neg)) continue;
        if (neg) {
            any_neg = true;
            double v[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) v[r] = X(r, i);
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const double lv = lam[i] * v[r];
#pragma unroll
                for (int c = 0; c <= r; ++c) Mp[pk(r, c)] = fma(-lv, v[c], Mp[pk(r, c)]);
            }
        }
    }
    if (!any_neg) return;
    // Hd[a][m + 1] = SG[a][m] / 2 for the three non-translation modes
    constexpr int SG[4][3] = {{1, 1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, 1}};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        // Ta[r][j] = sum_m SG[a][m] M'[(3m + r), j]
        double Ta[3][9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 9; ++j)
                Ta[r][j] = SG[a][0] * Mp[pk(r, j)] + SG[a][1] * Mp[pk(3 + r, j)] +
                           SG[a][2] * Mp[pk(6 + r, j)];
#pragma unroll
        for (int b = a; b < 4; ++b)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double h = 0.25 * (SG[b][0] * Ta[r][c] + SG[b][1] * Ta[r][3 + c] +
                                             SG[b][2] * Ta[r][6 + c]);
                    if (staged) {
                        staged[9 * up_index(a, b) + 3 * r + c] = (HT)h;
                    } else {
                        full[(3 * a + r) * 12 + 3 * b + c] = h;
                        if (a != b) full[(3 * b + c) * 12 + 3 * a + r] = h;
                    }
                }
    }
}

// phase 2 of the projection: one thread per queued stencil (the loop takes
// more than one trip only if the grid is smaller than the queue); subtracts
// sum_{lambda_t < -tau} lambda_t u_t u_t^T from its Hessian blocks
template <typename HT, int NT>
__global__ void __launch_bounds__(NT)
k_clamp(ElemLaunch L)
{
    extern __shared__ __align__(16) double Xs[];   // [81][NT]
    const SmemMat X{Xs + threadIdx.x, NT};
    const int count = min(*L.clamp_count, L.clamp_cap);
    // every thread of a block takes the same number of trips
    const int64_t span = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += span) {
        const int64_t idx = base + threadIdx.x;
        const unsigned live = __ballot_sync(0xffffffffu, idx < count);
        if (idx >= count) break;
        const ClampRef ref = L.clamp_ref[idx];
        const double* Mg = L.clamp_M + 45 * idx;
        double tau, fro;
        {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) {
                    const double v = Mg[pk(i, j)];
                    s = fma((i == j ? 1.0 : 2.0) * v, v, s);
                }
            fro = sqrt(s);
            tau = 1e-13 * fro;
        }
        double lam[9];
        const int k = eig9(Mg, X, lam, fro, sizeof(HT) == 4 ? SX_CLAMP_THETA32 : 1e-13, live);
        clamp_finish<HT>(L, ref, Mg, X, lam, k, tau, live);
    }
}

// The projection of a batched evaluation in split launches. The float part
// runs per queued stencil, writes its record and bins the stencil by k (the
// size of its N block, 0..9); the double parts then take the stencils bin by
// bin, so the 32 stencils of a warp share k: the refinement (k_clamp_refine,
// k = 1..3) and the block-restricted Jacobi (k_clamp_double, k >= 4 and what
// the refinement hands over), whose arithmetic is that of k_clamp. k = 0
// needs nothing (M positive definite by the float Gershgorin test).
// float part: one thread per queued stencil; its eigenvector matrix lives in
// shared memory ([81][NT + 1]: the odd stride keeps the copy-out free of
// bank conflicts), next to [NT][17] words of eigenvalues and slot order.
// The block's records are contiguous (record = queue position), so they are
// copied out by the whole block with coalesced stores.
constexpr int kClampFloatThreads = 128;
constexpr int clamp_float_smem(int nt) { return (81 * (nt + 1) + 17 * nt) * 4; }
// resident blocks per SM the float part is compiled for (a register cap;
// 4, i.e. 128 registers, measured slower on the 64^3 cube: projection 4.50
// -> 4.85 ms)
#ifndef SX_CLAMP_FLOAT_MINB
#define SX_CLAMP_FLOAT_MINB 1
#endif

template <int NT>
__global__ void __launch_bounds__(NT, SX_CLAMP_FLOAT_MINB)
k_clamp_float(ElemLaunch L)
{
    extern __shared__ __align__(16) float Xfs[];
    constexpr int XS = NT + 1;
    float* Ms = Xfs + 81 * XS;
    const int count = min(*L.clamp_count, L.clamp_cap);
    const int64_t base = (int64_t)blockIdx.x * NT;
    if (base >= count) return;   // the whole block
    const int64_t idx = base + threadIdx.x;
    if (idx < count) {
        const double* Mg = L.clamp_M + 45 * idx;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                const double v = Mg[pk(i, j)];
                s = fma((i == j ? 1.0 : 2.0) * v, v, s);
            }
        const double fro = sqrt(s);
        const int64_t cap = L.clamp_cap;
        const SmemXf Xf{Xfs + threadIdx.x, XS};
        float* ms = Ms + 17 * threadIdx.x;
        unsigned long long order = 0ull;
        const float delta = 1e-5f * (float)fro;
        int kneg = 0;   // eigenvalues below -delta
        int k = eig9_float_x(
            Mg, fro, Xf, [](int, int, float) {},
            [&](int slot, int c, float l) {
                ms[c] = l;
                order |= (unsigned long long)c << (4 * slot);
                kneg += (l < -delta) ? 1 : 0;
            });
        ms[9] = __uint_as_float((unsigned)order);
        ms[10] = __uint_as_float((unsigned)(order >> 32));
        // a non-finite matrix goes to the full double Jacobi, which reports it
        if (!isfinite(fro)) k = 9;
        ms[11] = __int_as_float(k);
        L.clamp_fro[idx] = fro;
        // bin: k, or for k >= 4 with 1..3 clearly negative modes the deflation
        // of those (a null space, as the barrier stencils' 4 structural
        // zeros, then needs no rotation; the rest is certified in double)
        const int bin = (SX_CLAMP_REFINE && SX_CLAMP_DEFL && k >= 4 && kneg >= 1 && kneg <= 3 &&
                         isfinite(fro))
                            ? kClampDefl + kneg
                            : k;
        // bucket slot: one atomic per (warp, bin) for the lanes that share it
        const unsigned peers = __match_any_sync(__activemask(), bin);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        int b0 = 0;
        if (lane == leader) b0 = atomicAdd(L.clamp_bucket_count + bin, __popc(peers));
        b0 = __shfl_sync(peers, b0, leader);
        const int pos = b0 + __popc(peers & ((1u << lane) - 1u));
        L.clamp_bucket[(int64_t)bin * cap + pos] = (int)idx;
    }
    __syncthreads();
    const int nrec = (int)(count - base < NT ? count - base : NT);
    float* dst = L.clamp_X + base * kClampRec;
    for (int g = threadIdx.x; g < nrec * kClampRec; g += NT) {
        const int t = g / kClampRec, j = g - t * kClampRec;
        float v = 0.0f;
        if (j < 81) v = Xfs[((j % 9) * 9 + j / 9) * XS + t];
        else if (j < 93) v = Ms[17 * t + (j - 81)];
        dst[g] = v;
    }
}

// the column of ascending-eigenvalue slot `slot` in a stencil's record
__device__ __forceinline__ unsigned long long rec_order(const float* rec)
{
    return (unsigned long long)__float_as_uint(__ldg(rec + 90)) |
           ((unsigned long long)__float_as_uint(__ldg(rec + 91)) << 32);
}
__device__ __forceinline__ int rec_col(unsigned long long order, int slot)
{
    return (int)((order >> (4 * slot)) & 15ull);
}

// resident threads per SM the double part is compiled for (a register cap:
// 65536 / this); 256 (two blocks of 128) measured best
#ifndef SX_CLAMP_MINB_THREADS
#define SX_CLAMP_MINB_THREADS 256
#endif
// one stencil of bin k (position jj) through the block-restricted double
// Jacobi
template <typename HT>
__device__ __forceinline__ void clamp_double_one(const ElemLaunch& L, const SmemMat& X, int k,
                                                 int jj, unsigned live)
{
    const int64_t cap = L.clamp_cap;
    const int64_t idx = L.clamp_bucket[(int64_t)k * cap + jj];
    const float* rec = L.clamp_X + idx * kClampRec;
    const unsigned long long order = rec_order(rec);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int col = rec_col(order, c);
#pragma unroll
        for (int r = 0; r < 9; ++r) X(r, c) = (double)__ldg(rec + 9 * col + r);
    }
    const ClampRef ref = L.clamp_ref[idx];
    const double* Mg = L.clamp_M + 45 * idx;
    const double fro = L.clamp_fro[idx];
    const double tau = 1e-13 * fro;
    double lam[9];
    eig9_double(Mg, X, lam, fro, sizeof(HT) == 4 ? SX_CLAMP_THETA32 : 1e-13, k, live);
    clamp_finish<HT>(L, ref, Mg, X, lam, k, tau, live);
}

template <typename HT, int NT>
__global__ void __launch_bounds__(NT, (SX_CLAMP_MINB_THREADS / NT) > 0 ? SX_CLAMP_MINB_THREADS / NT : 1)
k_clamp_double(ElemLaunch L)
{
    extern __shared__ __align__(16) double Xs[];   // [81][NT]
    const SmemMat X{Xs + threadIdx.x, NT};
    __shared__ int s_k, s_off;
    // work unit b -> (bucket, offset): buckets in order, ceil(count / NT)
    // units each; the grid loops over the units (with the N-block
    // refinement, k = 1..3 are done before, k = 0 needs nothing (M is
    // positive definite) and bin 9 goes to k_clamp_warp, so few stencils are
    // left here)
    for (int b0 = blockIdx.x;; b0 += gridDim.x) {
        if (threadIdx.x == 0) {
            int b = b0;
            s_k = -1;
            s_off = 0;
            for (int kk = SX_CLAMP_REFINE ? 4 : 0; kk < (SX_CLAMP_REFINE ? 9 : 10); ++kk) {
                const int nb = (L.clamp_bucket_count[kk] + NT - 1) / NT;
                if (b < nb) {
                    s_k = kk;
                    s_off = b * NT;
                    break;
                }
                b -= nb;
            }
        }
        __syncthreads();
        const int k = s_k;
        const int jj = s_off + threadIdx.x;
        __syncthreads();   // s_k, s_off read by all before thread 0 rewrites them
        if (k < 0) return;
        const int cntk = L.clamp_bucket_count[k];
        const unsigned live = __ballot_sync(0xffffffffu, jj < cntk);
        if (jj >= cntk) continue;
        clamp_double_one<HT>(L, X, k, jj, live);
    }
}

// N-block refinement of the stencils with k = 1..3 (sx_clamp.cuh). Pass 1
// takes bins 1..3, refines the k-column subspace and allows one
// correction; a stencil not certified by then goes to bin kClampPass2 + k.
// Pass 2 starts again from the float vectors and allows up to three
// corrections; a stencil not certified there goes to bin 9, the full double
// Jacobi. Pass 3 (the deflation) takes a stencil of k >= 4 whose float
// spectrum has k' = 1..3 eigenvalues below -delta: the k'-column subspace of
// those is refined the same way (up to three corrections) and the rest of
// M certified by a double LDL^T instead of rotated; a stencil not certified
// goes back to bin k. A stencil's result depends only on its own data. (A
// wider subspace in pass 2, max(k + 1, 3) columns, certified every stencil
// of a sample but measured slower on the 40^3 cube: 0.39 against 0.23 ms.)
template <typename HT, int K, int PASS>
__device__ __forceinline__ void clamp_refine_one(const ElemLaunch& L, int64_t idx, int k)
{
    const int64_t cap = L.clamp_cap;
    const float* rec = L.clamp_X + idx * kClampRec;
    const double* Mg = L.clamp_M + 45 * idx;
    const double fro = L.clamp_fro[idx];
    const double tau = 1e-13 * fro;
    const double thr = (sizeof(HT) == 4 ? SX_CLAMP_THETA32 : 1e-13) * fro;
    const double thr2 = thr * thr * (9 - K);
    // the record's eigenpairs in ascending order: slot q is column cq[q]
    const unsigned long long order = rec_order(rec);
    float mu[9];
    int cq[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        cq[q] = rec_col(order, q);
        mu[q] = __ldg(rec + 81 + cq[q]);
    }
    double V[9][K], R[9][K], B[K][K];
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
        for (int r = 0; r < 9; ++r) V[r][p] = f32_to_f64_bits(__ldg(rec + 9 * cq[p] + r));
    // the float vectors are orthonormal only to float precision: correct
    // once before the first certified residual
    refine_residual<K>(Mg, V, R, B);
    refine_correct<K>(rec, cq, mu, R, V);
    refine_residual<K>(Mg, V, R, B);
    constexpr int kMore = PASS == 1 ? 0 : 2;   // passes 2 and 3: up to three corrections
    bool conv = false;
#pragma unroll 1
    for (int it = 0;; ++it) {
        bool c = true;
#pragma unroll
        for (int p = 0; p < K; ++p) {
            double rn = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) rn = fma(R[r][p], R[r][p], rn);
            c = c && (rn <= thr2);
        }
        conv = c;
        if (conv || it >= kMore) break;
        refine_correct<K>(rec, cq, mu, R, V);
        refine_residual<K>(Mg, V, R, B);
    }
    // where a stencil goes that this pass does not finish: pass 1 -> its
    // second pass, pass 2 -> bin 9, pass 3 -> the bin of its N-block size
    const int bin_next = PASS == 1 ? kClampPass2 + k : PASS == 2 ? 9 : __float_as_int(__ldg(rec + 92));
    if (!conv) {
        const int pos = atomicAdd(L.clamp_bucket_count + bin_next, 1);
        L.clamp_bucket[(int64_t)bin_next * cap + pos] = (int)idx;
        return;
    }
    const ClampRef ref = L.clamp_ref[idx];
    bool ok = true;
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
        for (int j = 0; j < K; ++j) ok = ok && isfinite(B[p][j]);
    if (!ok) {
        atomicAdd(L.clamp_failed, 1);
        atomicExch(&L.scenes[ref.scene].sc->clamp_fail, 1);
        return;
    }
    // pass 3 (deflation): V holds the clearly negative modes only, the rest
    // of M (its near-null space and positive part) is certified instead of
    // rotated: M - V B V^T + s I positive definite (double LDL^T) means no
    // eigenvalue of the rest lies below -s. s = tau for an FP64 Hessian; for
    // an FP32 one 1e-6 ||M||_F: its exact zeros are spread over ~1e-7
    // ||M||_F by the float element math, and what lies above -1e-6 ||M||_F
    // is left unclamped (a change far inside that form's tolerance)
    const double rest_shift = sizeof(HT) == 4 ? 1e-6 * fro : tau;
    if (PASS == 3 && !refine_rest_pd<K>(Mg, V, B, rest_shift)) {
        const int pos = atomicAdd(L.clamp_bucket_count + bin_next, 1);
        L.clamp_bucket[(int64_t)bin_next * cap + pos] = (int)idx;
        return;
    }
    // B_-: the part of B below -tau
    if (!refine_negdef<K>(B, tau)) {
        refine_negpart<K>(B, tau, thr);
        bool any = false;
#pragma unroll
        for (int p = 0; p < K; ++p) any = any || B[p][p] != 0.0;
        if (!any) return;   // nothing below -tau: the blocks stay as they are
    }
    // U = 2 Ut: rows 3 a + r, the Hadamard inverse of V's mode rows (the
    // 1/2 of Hd is folded into B / 4)
    double U[12][K];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int p = 0; p < K; ++p) {
            const double y1 = V[r][p], y2 = V[3 + r][p], y3 = V[6 + r][p];
            const double a = y1 + y3, b = y1 - y3;
            U[r][p] = y2 + a;
            U[3 + r][p] = y2 - a;
            U[6 + r][p] = b - y2;
            U[9 + r][p] = -(b + y2);
        }
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
        for (int j = 0; j < K; ++j) B[p][j] *= 0.25;
    const SceneDev& S = L.scenes[ref.scene];
    const ElemBlock& Bk = S.blk[ref.blk];
    HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * (Bk.base + ref.e);
    double* full = L.out_H ? L.out_H + 144 * ref.e : nullptr;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        double UB[3][K];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < K; ++j) {
                double t = 0.0;
#pragma unroll
                for (int p = 0; p < K; ++p) t = fma(U[3 * a + r][p], B[p][j], t);
                UB[r][j] = t;
            }
#pragma unroll
        for (int b = a; b < 4; ++b)
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // (the correction d formed apart from the staged value:
                    // an FMA chain started from the loaded entry measured 3%
                    // slower, the load then on every chain's path)
                    double d = 0.0;
#pragma unroll
                    for (int j = 0; j < K; ++j) d = fma(UB[r][j], U[3 * b + c][j], d);
                    if (staged) {
                        HT* h = staged + 9 * up_index(a, b) + 3 * r + c;
                        *h = from_f64_bits<HT>(to_f64_bits(*h) - d);
                    } else {
                        const double h = full[(3 * a + r) * 12 + 3 * b + c] - d;
                        full[(3 * a + r) * 12 + 3 * b + c] = h;
                        if (a != b) full[(3 * b + c) * 12 + 3 * a + r] = h;
                    }
                }
    }
}

// Launch 1 takes bins 1..3 (pass 1); launch 2 takes the second-pass bins
// kClampPass2 + 1..3 and, in the same launch, the deflation bins
// kClampDefl + 1..3 (pass 3): a launch of its own over an empty bin cost
// 0.13 ms on the 64^3 cube. Work unit b -> (bin, offset) over the launch's
// bins in order; the grid loops.
template <typename HT, int LAUNCH, int NT>
__global__ void __launch_bounds__(NT)
k_clamp_refine(ElemLaunch L)
{
    __shared__ int s_bin, s_off;
    constexpr int nbins = LAUNCH == 1 ? 3 : (SX_CLAMP_DEFL ? 6 : 3);
    for (int b0 = blockIdx.x;; b0 += gridDim.x) {
        if (threadIdx.x == 0) {
            int b = b0;
            s_bin = -1;
            s_off = 0;
            for (int kk = 0; kk < nbins; ++kk) {
                const int bin = LAUNCH == 1 ? 1 + kk
                                            : (kk < 3 ? kClampPass2 + 1 + kk : kClampDefl + kk - 2);
                const int nb = (L.clamp_bucket_count[bin] + NT - 1) / NT;
                if (b < nb) {
                    s_bin = bin;
                    s_off = b * NT;
                    break;
                }
                b -= nb;
            }
        }
        __syncthreads();
        const int bin = s_bin;
        const int jj = s_off + threadIdx.x;
        __syncthreads();   // s_bin, s_off read by all before thread 0 rewrites them
        if (bin < 0) return;
        if (jj >= L.clamp_bucket_count[bin]) continue;
        const int64_t idx = L.clamp_bucket[(int64_t)bin * L.clamp_cap + jj];
        if (LAUNCH == 1) {
            const int k = bin;
            if (k == 1) clamp_refine_one<HT, 1, 1>(L, idx, k);
            else if (k == 2) clamp_refine_one<HT, 2, 1>(L, idx, k);
            else clamp_refine_one<HT, 3, 1>(L, idx, k);
        } else if (bin < kClampDefl) {
            const int k = bin - kClampPass2;
            if (k == 1) clamp_refine_one<HT, 1, 2>(L, idx, k);
            else if (k == 2) clamp_refine_one<HT, 2, 2>(L, idx, k);
            else clamp_refine_one<HT, 3, 2>(L, idx, k);
        } else {
            const int k = bin - kClampDefl;   // k', the negative modes
            if (k == 1) clamp_refine_one<HT, 1, 3>(L, idx, k);
            else if (k == 2) clamp_refine_one<HT, 2, 3>(L, idx, k);
            else clamp_refine_one<HT, 3, 3>(L, idx, k);
        }
    }
}

// Bin 9 (no certified small N block: the float Gershgorin test failed, or
// the refinement did not certify the stencil) holds few stencils, and one
// warp running a full double Jacobi for a thread's stencil takes a long
// time on this GPU (a warp's FP64 instruction occupies its SM quarter for
// 64 cycles). Here a warp takes one stencil and spreads the work over its
// lanes: the same algorithm as the k = 9 path of k_clamp_double (modified
// Gram-Schmidt of the float vectors, At = X^T M X, up to SX_F64_SWEEPS
// cyclic sweeps skipping |a_pq| <= theta ||M||_F, clamp below -tau,
// rewrite), with the sums in another order.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kClampWarpThreads = 128;

template <typename HT>
__global__ void __launch_bounds__(kClampWarpThreads)
k_clamp_warp(ElemLaunch L)
{
    constexpr int NW = kClampWarpThreads / 32;
    __shared__ double sX[NW][81], sY[NW][81], sA[NW][81];   // row-major r * 9 + c
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* X = sX[w];
    double* Y = sY[w];
    double* A = sA[w];
    const int64_t cap = L.clamp_cap;
    const int cnt = L.clamp_bucket_count[9];
    for (int j = blockIdx.x * NW + w; j < cnt; j += gridDim.x * NW) {
        const int64_t idx = L.clamp_bucket[9 * cap + j];
        const float* rec = L.clamp_X + idx * kClampRec;
        const unsigned long long order = rec_order(rec);
        const double* Mg = L.clamp_M + 45 * idx;
        const double fro = L.clamp_fro[idx];
        const double tau = 1e-13 * fro;
        const double thr = (sizeof(HT) == 4 ? SX_CLAMP_THETA32 : 1e-13) * fro;
        for (int e = lane; e < 81; e += 32) {
            const int r = e / 9, c = e - 9 * (e / 9);
            X[e] = (double)__ldg(rec + 9 * rec_col(order, c) + r);
        }
        __syncwarp();
        // modified Gram-Schmidt, column after column (lanes 0..8: the rows)
        for (int jc = 0; jc < 9; ++jc) {
            for (int ic = 0; ic < jc; ++ic) {
                const double d = warp_sum(lane < 9 ? X[lane * 9 + ic] * X[lane * 9 + jc] : 0.0);
                if (lane < 9) X[lane * 9 + jc] = fma(-d, X[lane * 9 + ic], X[lane * 9 + jc]);
                __syncwarp();
            }
            const double nn = warp_sum(lane < 9 ? X[lane * 9 + jc] * X[lane * 9 + jc] : 0.0);
            if (lane < 9) X[lane * 9 + jc] *= rsqrt(nn);
            __syncwarp();
        }
        // Y = M X, then At = X^T Y (the lower triangle, mirrored)
        for (int e = lane; e < 81; e += 32) {
            const int r = e / 9, c = e - 9 * (e / 9);
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < 9; ++q) t = fma(__ldg(Mg + pk(r, q)), X[q * 9 + c], t);
            Y[e] = t;
        }
        __syncwarp();
        for (int q = lane; q < 45; q += 32) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= q) ++i;
            const int c = q - i * (i + 1) / 2;
            double t = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) t = fma(X[r * 9 + i], Y[r * 9 + c], t);
            A[i * 9 + c] = t;
            A[c * 9 + i] = t;
        }
        __syncwarp();
        // cyclic sweeps (the whole warp on one pair at a time: lane r < 9
        // updates row r of A and of X)
        for (int sw = 0; sw < SX_F64_SWEEPS; ++sw)
            for (int p = 0; p < 8; ++p)
                for (int q = p + 1; q < 9; ++q) {
                    const double apq = A[p * 9 + q], app = A[p * 9 + p], aqq = A[q * 9 + q];
                    if (!(fabs(apq) > thr)) continue;   // the same on every lane
                    const float fpq = (float)apq;
                    const bool nz = fpq != 0.0f;
                    const float ft = jac_div((float)(aqq - app), nz ? 2.0f * fpq : 1.0f);
                    const float tt = jac_div(copysignf(1.0f, ft),
                                             fabsf(ft) + jac_sqrt1(fmaf(ft, ft, 1.0f)));
                    const double t = nz ? (double)tt : 0.0;
                    const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
                    double arp = 0.0, arq = 0.0, xp = 0.0, xq = 0.0;
                    if (lane < 9) {
                        arp = A[lane * 9 + p];
                        arq = A[lane * 9 + q];
                        xp = X[lane * 9 + p];
                        xq = X[lane * 9 + q];
                    }
                    __syncwarp();
                    if (lane < 9) {
                        if (lane != p && lane != q) {
                            const double nrp = fma(c, arp, -s * arq), nrq = fma(s, arp, c * arq);
                            A[lane * 9 + p] = nrp;
                            A[p * 9 + lane] = nrp;
                            A[lane * 9 + q] = nrq;
                            A[q * 9 + lane] = nrq;
                        }
                        X[lane * 9 + p] = fma(c, xp, -s * xq);
                        X[lane * 9 + q] = fma(s, xp, c * xq);
                    } else if (lane == 9) {
                        const double cc = c * c, ss = s * s, cs = c * s;
                        A[p * 9 + p] = fma(cc, app, fma(-2.0 * cs, apq, ss * aqq));
                        A[q * 9 + q] = fma(ss, app, fma(2.0 * cs, apq, cc * aqq));
                        const double npq = fma(cc - ss, apq, cs * (app - aqq));
                        A[p * 9 + q] = npq;
                        A[q * 9 + p] = npq;
                    }
                    __syncwarp();
                }
        double lam[9];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lam[i] = A[i * 9 + i];
            ok = ok && isfinite(lam[i]);
        }
        const ClampRef ref = L.clamp_ref[idx];
        if (!ok) {
            if (lane == 0) {
                atomicAdd(L.clamp_failed, 1);
                atomicExch(&L.scenes[ref.scene].sc->clamp_fail, 1);
            }
            continue;
        }
        bool any_neg = false;
#pragma unroll
        for (int i = 0; i < 9; ++i) any_neg = any_neg || lam[i] < -tau;
        if (!any_neg) continue;
        // M' = M - sum lambda v v^T (packed entries over the lanes, into Y)
        for (int q = lane; q < 45; q += 32) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= q) ++i;
            const int c = q - i * (i + 1) / 2;
            double m = __ldg(Mg + q);
#pragma unroll
            for (int l = 0; l < 9; ++l)
                if (lam[l] < -tau) m = fma(-lam[l] * X[i * 9 + l], X[c * 9 + l], m);
            Y[i * 9 + c] = m;
            Y[c * 9 + i] = m;
        }
        __syncwarp();
        // H' = (Hd kron I3) diag(0, M') (Hd kron I3)^T, the 10 upper blocks
        const SceneDev& S = L.scenes[ref.scene];
        const ElemBlock& Bk = S.blk[ref.blk];
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * (Bk.base + ref.e);
        double* full = L.out_H ? L.out_H + 144 * ref.e : nullptr;
        constexpr int SG[4][3] = {{1, 1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, 1}};
        for (int e = lane; e < 90; e += 32) {
            const int ab = e / 9, rc = e - 9 * (e / 9), r = rc / 3, c = rc - 3 * (rc / 3);
            int a = 0, b = 0;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = x; y < 4; ++y)
                    if (up_index(x, y) == ab) {
                        a = x;
                        b = y;
                    }
            double h = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int n = 0; n < 3; ++n)
                    h += (double)(SG[a][m] * SG[b][n]) * Y[(3 * m + r) * 9 + 3 * n + c];
            h *= 0.25;
            if (staged) {
                staged[9 * ab + rc] = (HT)h;
            } else {
                full[(3 * a + r) * 12 + 3 * b + c] = h;
                if (a != b) full[(3 * b + c) * 12 + 3 * a + r] = h;
            }
        }
        __syncwarp();
    }
}

// SM count of the current device (cached per device): the looping grids of
// the refinement's second pass and of the double part are sized by it
static int device_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        v = 152;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

cudaError_t launch_clamp(const ElemLaunch& L, cudaStream_t s)
{
    if (L.ntiles == 0 || !(L.level >= 2 && L.project)) return cudaSuccess;
    // the queue length stays on the device: the grid covers the largest
    // possible queue with one stencil per thread, and blocks past the actual
    // length exit at once. Short-lived blocks let work of higher-priority
    // streams (the serving lanes of small scenes) in between.
    const int cgrid = L.clamp_grid > 0 ? L.clamp_grid : 1;
    const int nt = (L.clamp_threads == 32 || L.clamp_threads == 128 || L.clamp_threads == 256)
                       ? L.clamp_threads
                       : 64;
    const int smem = 81 * 8 * nt + (L.share_sms ? clamp_share_pad(nt) : 0);
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (!bit || !(attr_done.load(std::memory_order_acquire) & bit)) {
        const void* fns[] = {(const void*)k_clamp<float, 32>, (const void*)k_clamp<float, 64>,
                             (const void*)k_clamp<float, 128>, (const void*)k_clamp<float, 256>,
                             (const void*)k_clamp<double, 32>, (const void*)k_clamp<double, 64>,
                             (const void*)k_clamp<double, 128>, (const void*)k_clamp<double, 256>,
                             (const void*)k_clamp_double<float, 32>,
                             (const void*)k_clamp_double<float, 64>,
                             (const void*)k_clamp_double<float, 128>,
                             (const void*)k_clamp_double<float, 256>,
                             (const void*)k_clamp_double<double, 32>,
                             (const void*)k_clamp_double<double, 64>,
                             (const void*)k_clamp_double<double, 128>,
                             (const void*)k_clamp_double<double, 256>};
        for (const void* f : fns)
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kClampMaxSmem);
        cudaFuncSetAttribute((const void*)k_clamp_float<kClampFloatThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             clamp_float_smem(kClampFloatThreads));
        attr_done.fetch_or(bit, std::memory_order_release);
    }
    const bool f32 = L.precision == SX_FP32;
    if (L.clamp_X) {
        // two launches: float part binned by k, then the double part per bucket
        const int64_t cap = L.clamp_cap;
        const int ga = (int)std::max<int64_t>(1, (cap + kClampFloatThreads - 1) / kClampFloatThreads);
        k_clamp_float<kClampFloatThreads>
            <<<ga, kClampFloatThreads, clamp_float_smem(kClampFloatThreads), s>>>(L);
        const int sms = device_sms();
        if (SX_CLAMP_REFINE) {
            // pass 1 covers its largest possible work in one trip; the
            // launch of pass 2 (a few percent of the stencils) and the
            // deflation (none on a tet mesh, most of a contact scene's
            // barrier stencils) loops over a grid of 8 blocks per SM
            const int gr = (int)std::max<int64_t>(1, (cap + 127) / 128 + 3);
            const int gr2 = std::min(gr, 8 * sms);
            if (f32) {
                k_clamp_refine<float, 1, 128><<<gr, 128, 0, s>>>(L);
                k_clamp_refine<float, 2, 128><<<gr2, 128, 0, s>>>(L);
            } else {
                k_clamp_refine<double, 1, 128><<<gr, 128, 0, s>>>(L);
                k_clamp_refine<double, 2, 128><<<gr2, 128, 0, s>>>(L);
            }
        }
        if (SX_CLAMP_REFINE) {
            // bin 9, a warp per stencil (grid-stride over the bin)
            const int gw = (int)std::min<int64_t>((cap + 3) / 4 + 1, 4 * sms);
            if (f32) k_clamp_warp<float><<<gw, kClampWarpThreads, 0, s>>>(L);
            else k_clamp_warp<double><<<gw, kClampWarpThreads, 0, s>>>(L);
        }
        // the double part loops over its units with at most 4 blocks per SM
        // (256 / nt more for smaller blocks); every stencil when the
        // refinement is off
        const int gfull = (int)std::max<int64_t>(1, (cap + nt - 1) / nt + 10);
        const int gb = SX_CLAMP_REFINE ? std::min(gfull, 4 * (256 / nt) * sms) : gfull;
        if (nt == 32) {
            if (f32) k_clamp_double<float, 32><<<gb, 32, smem, s>>>(L);
            else k_clamp_double<double, 32><<<gb, 32, smem, s>>>(L);
        } else if (nt == 128) {
            if (f32) k_clamp_double<float, 128><<<gb, 128, smem, s>>>(L);
            else k_clamp_double<double, 128><<<gb, 128, smem, s>>>(L);
        } else if (nt == 256) {
            if (f32) k_clamp_double<float, 256><<<gb, 256, smem, s>>>(L);
            else k_clamp_double<double, 256><<<gb, 256, smem, s>>>(L);
        } else {
            if (f32) k_clamp_double<float, 64><<<gb, 64, smem, s>>>(L);
            else k_clamp_double<double, 64><<<gb, 64, smem, s>>>(L);
        }
        return cudaGetLastError();
    }
    if (nt == 32) {
        if (f32) k_clamp<float, 32><<<cgrid, 32, smem, s>>>(L);
        else k_clamp<double, 32><<<cgrid, 32, smem, s>>>(L);
    } else if (nt == 128) {
        if (f32) k_clamp<float, 128><<<cgrid, 128, smem, s>>>(L);
        else k_clamp<double, 128><<<cgrid, 128, smem, s>>>(L);
    } else if (nt == 256) {
        if (f32) k_clamp<float, 256><<<cgrid, 256, smem, s>>>(L);
        else k_clamp<double, 256><<<cgrid, 256, smem, s>>>(L);
    } else {
        if (f32) k_clamp<float, 64><<<cgrid, 64, smem, s>>>(L);
        else k_clamp<double, 64><<<cgrid, 64, smem, s>>>(L);
    }
    return cudaGetLastError();
}

}  // namespace sx
