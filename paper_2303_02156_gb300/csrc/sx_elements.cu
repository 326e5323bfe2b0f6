// sx_elements.cu -- launches of the element kernel (instantiations for
// SNH tets alone and for SNH tets with hinges and barriers; the
// material-projection, other-density and high-order instantiations live in
// sx_elements_fproj.cu, sx_elements_models.cu and sx_elements_ho.cu), the
// contact-pair activity kernels, the friction lag and the lagged rotations
// of the co-rotational densities.
#include <cuda_runtime.h>

#include <algorithm>

#include "sx_elements.cuh"

namespace sx {

int elements_block_threads() { return kElemThreads; }
int clamp_block_threads() { return kClampThreads; }

const void* elements_kernel_snh(int kinds, bool f32)
{
    return kinds == 1 ? elements_kernel_ptr<1>(f32) : elements_kernel_ptr<7>(f32);
}

cudaError_t launch_elements_snh(int kinds, bool f32, const ElemLaunch& L, int grid, cudaStream_t s)
{
    if (kinds == 1) elements_launch<1>(f32, L, grid, s);
    else elements_launch<7>(f32, L, grid, s);
    return cudaGetLastError();
}


// Activation of point-triangle pairs at the state x (the classification
// and distance of Eq. 15's barrier in double): keep[e] = 1 when the pair
// contributes (0 < d < dhat) or is in an error state (d <= 0, so that the
// next evaluation still reports it), 0 when it is inactive (d >= dhat).
__global__ void k_pair_activity(const double* __restrict__ x, const int4* __restrict__ conn,
                                int64_t n, double dhat, int* keep)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int4 t = conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    double xr[12];
    double p0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) p0[i] = x[3 * (int64_t)nid[0] + i];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) xr[3 * a + i] = x[3 * (int64_t)nid[a] + i] - p0[i];
    BarrierOut<double> bo;
    const int st = barrier_eval<double>(xr, dhat, 0.0, 0, bo);
    keep[e] = st != 0 ? 1 : 0;
}

// order-preserving gather of the kept pairs (offsets: exclusive scan of keep)
__global__ void k_gather_pairs(const int4* __restrict__ conn, const int* __restrict__ keep,
                               const int* __restrict__ offsets, int64_t n, int4* out)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n || !keep[e]) return;
    out[offsets[e]] = conn[e];
}

cudaError_t launch_pair_activity(const double* x, const int4* conn, int64_t n, double dhat,
                                 int* keep, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_pair_activity<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(x, conn, n, dhat, keep);
    return cudaGetLastError();
}

cudaError_t launch_gather_pairs(const int4* conn, const int* keep, const int* offsets, int64_t n,
                                int4* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_gather_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(conn, keep, offsets, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ friction lag
// Lag of point-triangle pairs at the state x: the closest point of the
// triangle (the barrier's classification: the plane projection when its
// barycentrics are all >= 0, else the nearest clamped segment projection),
// its weights beta, d = |p - c|, fn = -b'(d) = kappa (2 (d - dhat) ln(d/dhat)
// + (d - dhat)^2 / d) for 0 < d < dhat (else 0), the unit normal (p - c)/d
// and a tangent basis: the coordinate axis least aligned with the normal,
// orthogonalized and normalized, then normal x that. Written as [13][n]:
// beta, T (two rows), fn, dx_lag = p - c.
__global__ void k_friction_lag(const double* __restrict__ x, const int4* __restrict__ conn,
                               int64_t n, double dhat, double kappa, double* __restrict__ lag)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int4 q = conn[e];
    const int nid[4] = {q.x, q.y, q.z, q.w};
    double t[3][3];   // triangle vertices relative to p
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            t[a][i] = x[3 * (int64_t)nid[a + 1] + i] - x[3 * (int64_t)nid[0] + i];
    double beta[3] = {0.0, 0.0, 0.0};
    bool face = false;
    {
        double E1[3], E2[3], ev[3], N[3], c1[3], c2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            E1[i] = t[1][i] - t[0][i];
            E2[i] = t[2][i] - t[0][i];
            ev[i] = -t[0][i];
        }
        cross3(E1, E2, N);
        const double w = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
        if (w > 0.0) {
            cross3(ev, E2, c1);
            cross3(E1, ev, c2);
            const double b1 = (c1[0] * N[0] + c1[1] * N[1] + c1[2] * N[2]) / w;
            const double b2 = (c2[0] * N[0] + c2[1] * N[1] + c2[2] * N[2]) / w;
            const double b0 = 1.0 - b1 - b2;
            if (b0 >= 0.0 && b1 >= 0.0 && b2 >= 0.0) {
                face = true;
                beta[0] = b0;
                beta[1] = b1;
                beta[2] = b2;
            }
        }
    }
    if (!face) {
        double best = 0.0, bt = 0.0;
        int bi = -1;
        for (int sgm = 0; sgm < 3; ++sgm) {
            const int iu = sgm, iw = (sgm + 1) % 3;
            double ee[3], EE[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ee[i] = -t[iu][i];
                EE[i] = t[iw][i] - t[iu][i];
            }
            const double bb = EE[0] * EE[0] + EE[1] * EE[1] + EE[2] * EE[2];
            double tt = bb > 0.0 ? (ee[0] * EE[0] + ee[1] * EE[1] + ee[2] * EE[2]) / bb : 0.0;
            tt = tt < 0.0 ? 0.0 : (tt > 1.0 ? 1.0 : tt);
            double dd = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double r = ee[i] - tt * EE[i];
                dd += r * r;
            }
            if (bi < 0 || dd < best) {
                best = dd;
                bt = tt;
                bi = sgm;
            }
        }
        beta[bi] = 1.0 - bt;
        beta[(bi + 1) % 3] = bt;
    }
    double r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = -(beta[0] * t[0][i] + beta[1] * t[1][i] + beta[2] * t[2][i]);
    const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double fn = 0.0;
    if (d > 0.0 && d < dhat) {
        const double dd = d - dhat;
        fn = kappa * (2.0 * dd * log(d / dhat) + dd * dd / d);
    }
    double nv[3] = {0.0, 0.0, 1.0};
    if (d > 0.0)
#pragma unroll
        for (int i = 0; i < 3; ++i) nv[i] = r[i] / d;
    const double a0 = fabs(nv[0]), a1 = fabs(nv[1]), a2 = fabs(nv[2]);
    const int ax = (a0 <= a1 && a0 <= a2) ? 0 : (a1 <= a2 ? 1 : 2);
    double t1[3], t2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t1[i] = (i == ax ? 1.0 : 0.0) - nv[ax] * nv[i];
    const double l1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) t1[i] /= l1;
    cross3(nv, t1, t2);
    double out[13] = {beta[0], beta[1], beta[2], t1[0], t1[1], t1[2], t2[0], t2[1], t2[2],
                      fn, r[0], r[1], r[2]};
#pragma unroll
    for (int k = 0; k < 13; ++k) lag[(int64_t)k * n + e] = out[k];
}

cudaError_t launch_friction_lag(const double* x, const int4* conn, int64_t n, double dhat,
                                double kappa, double* lag, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_friction_lag<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(x, conn, n, dhat, kappa, lag);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ lagged rotations
// R = U V^T of F = U diag(s) V^T (s descending) for every tet of a block:
// V from Jacobi on F^T F (made a rotation: v2 = v0 x v1), u0 = F v0 / |F v0|,
// u1 = F v1 with its u0 part removed, normalized, u2 = u0 x u1. For
// det F > 0 this is the rotation of the polar decomposition; for det F < 0
// the direction of the smallest singular value is flipped (the rotation
// nearest to F). F = 0 gives the identity; a rank-1 F completes u1 with the
// coordinate axis least aligned with u0.
__global__ void k_tet_rotations(const int4* __restrict__ conn, const double* __restrict__ x,
                                const double* __restrict__ Dminv, int64_t n,
                                double* __restrict__ Rout)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int4 t = conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    double F[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double f = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                f = fma(x[3 * (int64_t)nid[k + 1] + i] - x[3 * (int64_t)nid[0] + i],
                        Dminv[(int64_t)(k * 3 + j) * n + e], f);
            F[i * 3 + j] = f;
        }
    double A[6];   // F^T F packed lower
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            A[pk(i, j)] = F[0 * 3 + i] * F[0 * 3 + j] + F[1 * 3 + i] * F[1 * 3 + j] +
                          F[2 * 3 + i] * F[2 * 3 + j];
    double Q[9];
    jacobi3(A, Q);
    const double ev[3] = {A[0], A[2], A[5]};
    // order: i0 largest, i1 middle
    int i0 = 0, i1 = 1, i2 = 2;
    if (ev[i1] > ev[i0]) { const int tt = i0; i0 = i1; i1 = tt; }
    if (ev[i2] > ev[i0]) { const int tt = i0; i0 = i2; i2 = tt; }
    if (ev[i2] > ev[i1]) { const int tt = i1; i1 = i2; i2 = tt; }
    double v0[3], v1[3], v2[3], u0[3], u1[3], u2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        v0[r] = Q[3 * r + i0];
        v1[r] = Q[3 * r + i1];
    }
    cross3(v0, v1, v2);
    matvec3(F, v0, u0);
    matvec3(F, v1, u1);
    double R[9];
    const double n0 = sqrt(u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);
    if (!(n0 > 0.0)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) u0[r] /= n0;
        double d = u0[0] * u1[0] + u0[1] * u1[1] + u0[2] * u1[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] -= d * u0[r];
        double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
        if (!(n1 > 1e-14 * n0)) {
            // rank 1: the axis least aligned with u0
            const double a0 = fabs(u0[0]), a1 = fabs(u0[1]), a2 = fabs(u0[2]);
            const int ax = (a0 <= a1 && a0 <= a2) ? 0 : (a1 <= a2 ? 1 : 2);
#pragma unroll
            for (int r = 0; r < 3; ++r) u1[r] = (r == ax ? 1.0 : 0.0) - u0[ax] * u0[r];
            n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] /= n1;
        cross3(u0, u1, u2);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                R[i * 3 + j] = u0[i] * v0[j] + u1[i] * v1[j] + u2[i] * v2[j];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) Rout[(int64_t)k * n + e] = R[k];
}

cudaError_t launch_tet_rotations(const int4* conn, const double* x, const double* Dminv,
                                 int64_t n, double* R, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_tet_rotations<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(conn, x, Dminv, n, R);
    return cudaGetLastError();
}

const void* elements_kernel(int precision, int variant)
{
    const bool f = precision == SX_FP32;
    switch (variant) {
    case 1: return elements_kernel_snh(1, f);
    case 2: return elements_kernel_fproj(15, f);
    case 3: return elements_kernel_fproj(9, f);
    case 4: return elements_kernel_models(25, f);
    case 5: return elements_kernel_models(63, f);
    case 6: return elements_kernel_ho(64, f);
    case 7: return elements_kernel_ho(127, f);
    default: return elements_kernel_snh(7, f);
    }
}

int elements_variant(int kinds, int project)
{
    // high-order tets: alone, or with every other kind
    if (kinds & 64) return (kinds & ~64) ? 7 : 6;
    // tets of the other densities or friction: one instantiation with the
    // material projection compiled in, for tets alone or every kind
    if (kinds & (16 | 32)) return (kinds & (2 | 4 | 32)) ? 5 : 4;
    const bool snh_only = kinds == 1;
    return project == 2 ? (snh_only ? 3 : 2) : (snh_only ? 1 : 0);
}

cudaError_t launch_elements(const ElemLaunch& L, int grid, cudaStream_t s)
{
    if (L.ntiles == 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(L.queue, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    if (L.level >= 2 && L.project) {
        err = cudaMemsetAsync(L.clamp_count, 0, sizeof(int), s);
        if (err == cudaSuccess && L.clamp_bucket_count)
            err = cudaMemsetAsync(L.clamp_bucket_count, 0, kClampBins * sizeof(int), s);
        if (err != cudaSuccess) return err;
    }
    const bool f = L.precision == SX_FP32;
    switch (elements_variant(L.kinds, L.level >= 2 ? L.project : 0)) {
    case 1: return launch_elements_snh(1, f, L, grid, s);
    case 2: return launch_elements_fproj(15, f, L, grid, s);
    case 3: return launch_elements_fproj(9, f, L, grid, s);
    case 4: return launch_elements_models(25, f, L, grid, s);
    case 5: return launch_elements_models(63, f, L, grid, s);
    case 6: return launch_elements_ho(64, f, L, grid, s);
    case 7: return launch_elements_ho(127, f, L, grid, s);
    default: return launch_elements_snh(7, f, L, grid, s);
    }
}

}  // namespace sx
