// sx_clamp.cuh -- FP64 projection of a 4-node stencil Hessian to PSD
// (§5.2 "Projection to positive semi-definiteness"; Algorithm 1 ProjectToPD).
//
// A 4-node stencil energy that is invariant under translation has a
// 12x12 Hessian H with the 3 translations in its null space. In the
// orthonormal Hadamard basis of the four nodes, y = (Hd kron I3) x with
// Hd = 1/2 [[1,1,1,1],[1,-1,1,-1],[1,1,-1,-1],[1,-1,-1,1]], H becomes
// diag(0_3, M) with M the 9x9 Hessian of the three non-translation modes.
// Clamping the eigenvalues of H at zero is therefore the same as clamping
// those of M: proj(H) = H - sum_{lambda_i < 0} lambda_i u_i u_i^T with
// u_i = (Hd kron I3)(0, v_i) and (lambda_i, v_i) the negative eigenpairs
// of M. The 9x9 problem is solved in double precision in two phases:
//   1. (element kernel) shifted LDL^T of M + tau I, tau = 1e-13 ||M||_F:
//      if it succeeds the stencil is left as is (the change is at most
//      tau); otherwise M is queued for phase 2;
//   2. (clamp kernel, one thread per queued M) cyclic Jacobi in float from
//      the identity (float is ~60x faster than double on this part); the
//      approximate eigenpairs are ordered by ascending eigenvalue, and the
//      first k (eigenvalue below delta = 1e-5 ||M||_F) form the block N
//      that can hold negative eigenvalues. In double: modified Gram-Schmidt
//      of the float eigenvectors, At = X^T M X (nearly diagonal), and
//      Jacobi sweeps on At, accumulated into X, that rotate only the pairs
//      (p, q) with p in N (p < k) and skip a rotation whose |a_pq| is at
//      most theta ||M||_F: theta = 1e-13 for an FP64 Hessian; 1e-9 for an
//      FP32 one (its entries carry ~6e-8 relative rounding, which also
//      spreads its exactly-zero eigenvalues over ~1e-7 ||M||, and the
//      result is stored in float). Eigenvalues of the N block below -tau
//      are clamped: M' = M - sum of lambda v v^T over them, and the
//      stencil's Hessian is rewritten as (Hd kron I3) diag(0, M')
//      (Hd kron I3)^T.
//   For k = 1..3 (nearly every queued SNH tet: its negative modes are
//   the rotational ones) the double part instead refines the k-column
//   subspace alone, with a certified residual (see "N-block refinement"
//   below); the Jacobi described above is the path of every other k and of
//   a stencil the refinement does not certify.
//   Accuracy: clamping at zero is 1-Lipschitz in the Frobenius norm on
//   symmetric matrices, so the projection is off by at most about twice the
//   Frobenius norm of the N-N and N-P off-diagonal entries left in At
//   (each at most theta ||M||_F once a sweep skips them all). The P block
//   is left as it is: its eigenvalues are above delta minus the float
//   error, which a Gershgorin test on the float matrix confirms (else k =
//   9, a full Jacobi). A rotation runs for the warp when any of its lanes
//   needs it, and a lane that does not keeps its entries unchanged, so each
//   stencil's result does not depend on which stencils share its warp.
// Matrices are kept packed (lower triangle, 45 entries) and every loop is
// unrolled so they live in registers; the eigenvector matrix lives in
// shared memory. Jacobi is the textbook symmetric Schur method (Golub &
// Van Loan, ch. 8); the result, a spectral function of H, is unique even
// where eigenvectors are not.
#pragma once

#include <float.h>
#include <math.h>

namespace sx {

#ifndef SX_F64_SWEEPS
#define SX_F64_SWEEPS 3
#endif
// rotation skip threshold (relative to ||M||_F) for a Hessian computed in FP32
#ifndef SX_CLAMP_THETA32
#define SX_CLAMP_THETA32 1e-9
#endif

// The float Jacobi angle only decides how far a rotation goes (every
// rotation is exactly orthogonal in the precision it is applied in, and the
// double sweeps correct what the float ones leave), so it is computed with
// the approximate float division and square root (about 2 ulp) instead of
// the correctly rounded ones, which are long instruction sequences on the
// serial chain of a Jacobi sweep.
#ifndef SX_CLAMP_FAST_F32
#define SX_CLAMP_FAST_F32 1
#endif
__device__ __forceinline__ float jac_div(float a, float b)
{
    return SX_CLAMP_FAST_F32 ? __fdividef(a, b) : a / b;
}
// sqrt of x >= 1 (x may be +inf: tau^2 + 1 overflows when a_pq is tiny;
// x rsqrt(x) would give inf * 0 there)
__device__ __forceinline__ float jac_sqrt1(float x)
{
    return (SX_CLAMP_FAST_F32 && x <= 1e36f) ? x * rsqrtf(x) : sqrtf(x);
}

// packed lower-triangle index of (i, j), any order
__host__ __device__ constexpr int pk(int i, int j)
{
    return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// 1/2 Hadamard columns c = 1..3 applied to node quantities (a = 0..3)
// y_c = sum_a Hd[a][c] x_a
template <typename T>
__device__ __forceinline__ void had_fwd(const T x0, const T x1, const T x2, const T x3,
                                        T& y1, T& y2, T& y3)
{
    y1 = T(0.5) * ((x0 - x1) + (x2 - x3));
    y2 = T(0.5) * ((x0 + x1) - (x2 + x3));
    y3 = T(0.5) * ((x0 - x1) - (x2 - x3));
}
// x_a = sum_{c=1..3} Hd[a][c] y_c  (the translation component y0 = 0)
template <typename T>
__device__ __forceinline__ void had_inv(const T y1, const T y2, const T y3, T& x0, T& x1,
                                        T& x2, T& x3)
{
    x0 = T(0.5) * (y1 + y2 + y3);
    x1 = T(0.5) * (y2 - y1 - y3);
    x2 = T(0.5) * (y1 - y2 - y3);
    x3 = T(0.5) * (y3 - y1 - y2);
}

__device__ __forceinline__ double fro9(const double (&A)[45])
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) s = fma((i == j ? 1.0 : 2.0) * A[pk(i, j)], A[pk(i, j)], s);
    return sqrt(s);
}

// Phase 1: true when M + tau I is positive definite (LDL^T without
// pivoting succeeds), tau = 1e-13 ||M||_F. M is not modified.
__device__ __forceinline__ bool psd_by_ldlt(const double (&M)[45])
{
    const double fro = fro9(M);
    if (fro == 0.0) return true;
    const double tau = 1e-13 * fro;
    double L[45];
    double dg[9];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        double s = M[pk(j, j)] + tau;
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[pk(j, k)] * L[pk(j, k)] * dg[k];
        pd = pd && (s > 0.0);
        dg[j] = s;
        const double inv = 1.0 / s;
#pragma unroll
        for (int i = j + 1; i < 9; ++i) {
            double t = M[pk(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[pk(i, k)] * L[pk(j, k)] * dg[k];
            L[pk(i, j)] = t * inv;
        }
    }
    return pd;
}

// Phase 1 pre-test in float, with a margin delta = 1e-4 ||M||_F that covers
// the backward error of a float LDL^T of a 9x9 (about 9 * 2^-24 times a
// small constant, relative to ||M||): LDL^T of M - delta I succeeding
// proves M positive definite (+1); LDL^T of M + delta I failing proves an
// eigenvalue below -delta/2 (-1). Both decide as the double test would;
// 0 leaves the decision to it.
__device__ __forceinline__ bool ldlt_f32_pd(const float (&A)[45], float shift)
{
    float L[45];
    float dg[9];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        float s = A[pk(j, j)] + shift;
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[pk(j, k)] * L[pk(j, k)] * dg[k];
        pd = pd && (s > 0.0f);
        dg[j] = s;
        const float inv = 1.0f / s;
#pragma unroll
        for (int i = j + 1; i < 9; ++i) {
            float t = A[pk(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[pk(i, k)] * L[pk(j, k)] * dg[k];
            L[pk(i, j)] = t * inv;
        }
    }
    return pd;
}

// double -> float with the mantissa truncated (toward zero), built from the
// bit fields on the integer pipe: on this GPU a hardware conversion issues
// on the FP64 pipe, which the element kernels saturate. Magnitudes below
// the normal float range give a signed zero; above it (and inf, NaN) a NaN,
// which leaves the pre-test undecided. The truncation (at most 2^-23
// relative) is far inside the pre-test's margin.
__device__ __forceinline__ float f64_to_f32_trunc(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned ex = (hi >> 20) & 0x7FFu;
    unsigned f;
    if (ex <= 896u) f = 0u;
    else if (ex >= 1151u) f = 0x7FC00000u;
    else f = ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return __uint_as_float((hi & 0x80000000u) | f);
}

// double -> float rounded to nearest (ties to even) from the bit fields on
// the integer pipe: the 29 dropped mantissa bits are rounded into the kept
// ones (a carry runs on into the exponent, as it should); results outside
// the normal float range as in f64_to_f32_trunc
__device__ __forceinline__ float f64_to_f32_rn(double d)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sg = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned ex0 = (unsigned)(b >> 52) & 0x7FFu;
    if (ex0 == 0x7FFu) return __uint_as_float(sg | 0x7FC00000u);
    b += 0x0FFFFFFFull + ((b >> 29) & 1ull);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned ex = (hi >> 20) & 0x7FFu;
    unsigned f;
    if (ex <= 896u) f = 0u;
    else if (ex >= 1151u) f = 0x7FC00000u;
    else f = ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return __uint_as_float(sg | f);
}

// float -> double (exact) from the bit fields on the integer pipe; a
// subnormal float takes the hardware conversion
__device__ __forceinline__ double f32_to_f64_bits(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned ex = (u >> 23) & 0xFFu, mt = u & 0x7FFFFFu, sg = u & 0x80000000u;
    if (ex == 0u && mt != 0u) return (double)x;
    const unsigned e64 = ex == 0u ? 0u : (ex == 255u ? 2047u : ex + 896u);
    return __hiloint2double((int)(sg | (e64 << 20) | (mt >> 3)), (int)(mt << 29));
}
__device__ __forceinline__ double to_f64_bits(float x) { return f32_to_f64_bits(x); }
__device__ __forceinline__ double to_f64_bits(double x) { return x; }
// a double result stored as HT (float: rounded to nearest on the integer pipe)
template <typename HT>
__device__ __forceinline__ HT from_f64_bits(double x);
template <>
__device__ __forceinline__ double from_f64_bits<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64_bits<float>(double x) { return f64_to_f32_rn(x); }

__device__ __forceinline__ int psd_class_f32(const double (&M)[45])
{
    float A[45];
    float f2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const float v = f64_to_f32_trunc(M[pk(i, j)]);
            A[pk(i, j)] = v;
            f2 = fmaf((i == j ? 1.0f : 2.0f) * v, v, f2);
        }
    const float delta = 1e-4f * sqrtf(f2);
    if (!(delta > 0.0f) || !isfinite(delta)) return 0;
    if (ldlt_f32_pd(A, -delta)) return 1;
    if (!ldlt_f32_pd(A, delta)) return -1;
    return 0;
}

// ---------------------------------------------------------------- phase 2
// Cyclic Jacobi (symmetric Schur rotations, Golub & Van Loan 8.5) on the
// packed 9x9 A with the rotations accumulated into X (row-major, column c =
// eigenvector c). One sweep visits the 36 pairs (p, q) in a fixed order;
// every loop is unrolled and there is no data-dependent control flow, so a
// warp runs its 32 stencils in lockstep.

// The float eigenvector matrix, row-major (column c = eigenvector c): in
// registers (a per-thread array) or in shared memory laid out [81][threads]
// (fewer registers, more resident warps for the float Jacobi's serial
// chains).
struct RegXf {
    float (&a)[81];
    __device__ __forceinline__ float& operator()(int r, int c) const { return a[r * 9 + c]; }
};
struct SmemXf {
    float* base;
    int stride;
    __device__ __forceinline__ float& operator()(int r, int c) const
    {
        return base[(r * 9 + c) * stride];
    }
};

// float sweep: exact float angle, a_pq set to zero
template <typename XF>
__device__ __forceinline__ void jacobi_sweep_f32(float (&A)[45], const XF& X)
{
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = p + 1; q < 9; ++q) {
            const float apq = A[pk(p, q)], app = A[pk(p, p)], aqq = A[pk(q, q)];
            const bool nz = apq != 0.0f;
            const float tau = jac_div(aqq - app, nz ? 2.0f * apq : 1.0f);
            const float tt = jac_div(copysignf(1.0f, tau),
                                     fabsf(tau) + jac_sqrt1(fmaf(tau, tau, 1.0f)));
            const float t = nz ? tt : 0.0f;
            const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
            A[pk(p, p)] = app - t * apq;
            A[pk(q, q)] = aqq + t * apq;
            A[pk(p, q)] = 0.0f;
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                if (r == p || r == q) continue;
                const float arp = A[pk(r, p)], arq = A[pk(r, q)];
                A[pk(r, p)] = c * arp - s * arq;
                A[pk(r, q)] = s * arp + c * arq;
            }
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const float xp = X(r, p), xq = X(r, q);
                X(r, p) = c * xp - s * xq;
                X(r, q) = s * xp + c * xq;
            }
        }
}

// Accessor for a per-thread 9x9 double matrix in shared memory laid out
// [81][threads] so that a warp's accesses to the same entry are contiguous.
struct SmemMat {
    double* base;
    int stride;
    __device__ __forceinline__ double& operator()(int r, int c) const
    {
        return base[(r * 9 + c) * stride];
    }
};

// double sweep: the angle comes from float arithmetic (it only decides how
// much a_pq shrinks), the rotation (c, s = t c with c = 1/sqrt(1+t^2)) and
// the 2x2 update are exact in double, so A stays similar to M to working
// precision. Pairs (p, q), p < q, with p >= k or |a_pq| <= thr are left
// alone (their entries keep their values bit for bit); the warp skips a
// pair that none of its lanes (mask live) needs.
__device__ __forceinline__ void jacobi_sweep_f64(double (&A)[45], const SmemMat& X, int k,
                                                 double thr, unsigned live)
{
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = p + 1; q < 9; ++q) {
            const double apq = A[pk(p, q)], app = A[pk(p, p)], aqq = A[pk(q, q)];
            const bool need = (p < k) && (fabs(apq) > thr);
            if (!__any_sync(live, need)) continue;
            const float fpq = (float)apq;
            const bool nz = fpq != 0.0f;
            const float tau = jac_div((float)(aqq - app), nz ? 2.0f * fpq : 1.0f);
            const float tt = jac_div(copysignf(1.0f, tau),
                                     fabsf(tau) + jac_sqrt1(fmaf(tau, tau, 1.0f)));
            const double t = nz ? (double)tt : 0.0;
            const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
            const double cc = c * c, ss = s * s, cs = c * s;
            const double npp = fma(cc, app, fma(-2.0 * cs, apq, ss * aqq));
            const double nqq = fma(ss, app, fma(2.0 * cs, apq, cc * aqq));
            const double npq = fma(cc - ss, apq, cs * (app - aqq));
            A[pk(p, p)] = need ? npp : app;
            A[pk(q, q)] = need ? nqq : aqq;
            A[pk(p, q)] = need ? npq : apq;
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                if (r == p || r == q) continue;
                const double arp = A[pk(r, p)], arq = A[pk(r, q)];
                const double nrp = fma(c, arp, -s * arq), nrq = fma(s, arp, c * arq);
                A[pk(r, p)] = need ? nrp : arp;
                A[pk(r, q)] = need ? nrq : arq;
            }
            if (need) {
#pragma unroll
                for (int r = 0; r < 9; ++r) {
                    const double xp = X(r, p), xq = X(r, q);
                    X(r, p) = fma(c, xp, -s * xq);
                    X(r, q) = fma(s, xp, c * xq);
                }
            }
        }
}

// Phase 2, float part. Mg: packed 9x9 (double, global memory); fro =
// ||M||_F. Cyclic Jacobi in float from the identity, then the eigenvector
// columns ordered by ascending float eigenvalue: put(r, slot, value) stores
// entry r of the column that lands in `slot`. Returns k, the number of
// eigenvalues below delta = 1e-5 ||M||_F (9 when a Gershgorin test on the
// float matrix cannot confirm that the rest is a positive definite block).
// putl(slot, c, value) receives the float eigenvalue of column c, which
// lands in `slot`.
struct NoPutL {
    __device__ __forceinline__ void operator()(int, int, float) const {}
};
template <typename XF, typename Put, typename PutL = NoPutL>
__device__ __forceinline__ int eig9_float_x(const double* __restrict__ Mg, double fro, const XF& Xf,
                                            Put put, PutL putl = PutL())
{
    int k = 0;
    float A[45];
#pragma unroll
    for (int i = 0; i < 45; ++i) A[i] = (float)Mg[i];
#pragma unroll
    for (int i = 0; i < 81; ++i) Xf(i / 9, i % 9) = (i % 10 == 0) ? 1.0f : 0.0f;
    // (a round-robin pair order, four independent rotations at a time,
    // measured the same on the 64^3 cube: 4.475 against 4.492 ms per
    // projection; the cyclic order stays)
#pragma unroll 1
    for (int sw = 0; sw < 5; ++sw) jacobi_sweep_f32(A, Xf);
    const float delta = 1e-5f * (float)fro;
    bool pblock_ok = true;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float lc = A[pk(c, c)];
        int rank = 0;
        float rad = 0.0f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            if (j == c) continue;
            const float lj = A[pk(j, j)];
            rank += (lj < lc || (lj == lc && j < c)) ? 1 : 0;
            rad += (lj >= delta) ? fabsf(A[pk(c, j)]) : 0.0f;
        }
        k += (lc < delta) ? 1 : 0;
        // Gershgorin disc of the P block, with half of delta to spare
        if (lc >= delta) pblock_ok = pblock_ok && (lc - rad > 0.5f * delta);
#pragma unroll
        for (int r = 0; r < 9; ++r) put(r, rank, Xf(r, c));
        putl(rank, c, lc);
    }
    return pblock_ok ? k : 9;
}

// the same with the float eigenvectors in registers
template <typename Put>
__device__ __forceinline__ int eig9_float(const double* __restrict__ Mg, double fro, Put put)
{
    float a[81];
    return eig9_float_x(Mg, fro, RegXf{a}, put);
}

// Phase 2, double part: X (shared memory, columns ordered as above) is
// re-orthonormalized, At = X^T M X formed and the N-block rows rotated. On
// return the first k columns of X are eigenvectors of M with eigenvalues
// lam[0..k-1]; the other columns span an invariant subspace on which M is
// positive definite (lam[k..8] are then the diagonal of that block).
__device__ __forceinline__ void eig9_double(const double* __restrict__ Mg, const SmemMat& X,
                                            double (&lam)[9], double fro, double theta, int k,
                                            unsigned live)
{
    // re-orthonormalize in double (modified Gram-Schmidt; X is already
    // orthogonal to float precision, so one pass suffices)
#pragma unroll
    for (int j = 0; j < 9; ++j) {
#pragma unroll
        for (int i = 0; i < j; ++i) {
            double d = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) d = fma(X(r, i), X(r, j), d);
#pragma unroll
            for (int r = 0; r < 9; ++r) X(r, j) = fma(-d, X(r, i), X(r, j));
        }
        double nn = 0.0;
#pragma unroll
        for (int r = 0; r < 9; ++r) nn = fma(X(r, j), X(r, j), nn);
        const double inv = rsqrt(nn);
#pragma unroll
        for (int r = 0; r < 9; ++r) X(r, j) *= inv;
    }
    // At = X^T M X (nearly diagonal), then double Jacobi sweeps on the rows
    // of the N block
    double At[45];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        double y[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 9; ++c) s = fma(__ldg(Mg + pk(r, c)), X(c, j), s);
            y[r] = s;
        }
#pragma unroll
        for (int i = j; i < 9; ++i) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) s = fma(X(r, i), y[r], s);
            At[pk(i, j)] = s;
        }
    }
    const double thr = theta * fro;
#pragma unroll 1
    for (int sw = 0; sw < SX_F64_SWEEPS; ++sw) jacobi_sweep_f64(At, X, k, thr, live);
#pragma unroll
    for (int i = 0; i < 9; ++i) lam[i] = At[pk(i, i)];
}

// Both parts for one stencil (the eigenvector matrix X in shared memory).
__device__ __forceinline__ int eig9(const double* __restrict__ Mg, const SmemMat& X,
                                    double (&lam)[9], double fro, double theta, unsigned live)
{
    const int k = eig9_float(Mg, fro, [&](int r, int slot, float v) { X(r, slot) = (double)v; });
    eig9_double(Mg, X, lam, fro, theta, k, live);
    return k;
}

// ------------------------------------------------- N-block refinement (k <= 3)
// For a small N block the double part need not re-orthonormalize and
// rotate the whole 9x9: only the invariant subspace of the k lowest
// eigenvalues enters the clamp. It is refined as a subspace (Rayleigh-Ritz
// with a first-order correction, Golub & Van Loan 8.1, 8.2):
//   V = the k float eigenvectors of N (double), W = M V, B = V^T W (k x k),
//   R = W - V B, the part of M V outside span(V). With V orthonormal, V
//   spans an invariant subspace of M to within ||R||. The correction
//   v_p -= sum_{q in P} x_q (x_q . r_p) / (mu_q - mu_p), over the float
//   eigenpairs (mu_q, x_q) of the P block, removes R to first order; it only
//   has to be as accurate as float (it moves V by ~1e-7), so it runs in
//   float arithmetic. V is then re-orthonormalized (modified Gram-Schmidt)
//   and R recomputed in double, which certifies the result: a stencil is
//   done once ||r_p|| <= theta ||M||_F sqrt(9 - k) for every column p (the
//   same bound as k (9 - k) couplings of at most theta ||M||_F each).
// Then M' = M - V B_- V^T, with B_- the part of B below -tau (B itself when
// -B - tau I is positive definite, else from a small Jacobi on B), and the
// stencil's blocks become H - Ut B_- Ut^T with Ut = (Hd kron I3)(0; V).
// A stencil that is not certified after its allowed corrections is handed
// to the full double Jacobi (k = 9). Every step is per lane, so a stencil's
// result does not depend on the other stencils of its warp.

template <int K>
__device__ __forceinline__ void refine_mgs(double (&V)[9][K])
{
#pragma unroll
    for (int p = 0; p < K; ++p) {
#pragma unroll
        for (int j = 0; j < p; ++j) {
            double d = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) d = fma(V[r][j], V[r][p], d);
#pragma unroll
            for (int r = 0; r < 9; ++r) V[r][p] = fma(-d, V[r][j], V[r][p]);
        }
        double nn = 0.0;
#pragma unroll
        for (int r = 0; r < 9; ++r) nn = fma(V[r][p], V[r][p], nn);
        const double inv = rsqrt(nn);
#pragma unroll
        for (int r = 0; r < 9; ++r) V[r][p] *= inv;
    }
}

// W = M V, B = V^T W (symmetric: the lower triangle, mirrored), R = W - V B
// (R returned in place of W)
template <int K>
__device__ __forceinline__ void refine_residual(const double* __restrict__ Mg,
                                                const double (&V)[9][K], double (&R)[9][K],
                                                double (&B)[K][K])
{
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        double mr[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) mr[c] = __ldg(Mg + pk(r, c));
#pragma unroll
        for (int p = 0; p < K; ++p) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 9; ++c) s = fma(mr[c], V[c][p], s);
            R[r][p] = s;
        }
    }
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
        for (int j = 0; j <= p; ++j) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) s = fma(V[r][p], R[r][j], s);
            B[p][j] = s;
            B[j][p] = s;
        }
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int p = 0; p < K; ++p) {
            double s = R[r][p];
#pragma unroll
            for (int j = 0; j < K; ++j) s = fma(-V[r][j], B[j][p], s);
            R[r][p] = s;
        }
}

// first-order correction of V from the float eigenpairs of the P block
// (rec: the stencil's record, the eigenvector of ascending slot q at
// rec[9 cq[q]]; mu: the eigenvalues by slot)
template <int K>
__device__ __forceinline__ void refine_correct(const float* __restrict__ rec, const int (&cq)[9],
                                               const float (&mu)[9], const double (&R)[9][K],
                                               double (&V)[9][K])
{
    float rf[9][K], dv[9][K];
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int p = 0; p < K; ++p) {
            rf[r][p] = f64_to_f32_trunc(R[r][p]);
            dv[r][p] = 0.0f;
        }
#pragma unroll
    for (int q = K; q < 9; ++q) {
        float xq[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) xq[r] = __ldg(rec + 9 * cq[q] + r);
#pragma unroll
        for (int p = 0; p < K; ++p) {
            float c = 0.0f;
#pragma unroll
            for (int r = 0; r < 9; ++r) c = fmaf(xq[r], rf[r][p], c);
            const float z = __fdividef(c, mu[q] - mu[p]);
#pragma unroll
            for (int r = 0; r < 9; ++r) dv[r][p] = fmaf(xq[r], z, dv[r][p]);
        }
    }
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int p = 0; p < K; ++p) V[r][p] -= f32_to_f64_bits(dv[r][p]);
    refine_mgs<K>(V);
}

// true when -B - tau I is positive definite (every eigenvalue of B below
// -tau): LDL^T without pivoting
template <int K>
__device__ __forceinline__ bool refine_negdef(const double (&B)[K][K], double tau)
{
    double L[K][K], dg[K];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double s = -B[j][j] - tau;
#pragma unroll
        for (int m = 0; m < j; ++m) s -= L[j][m] * L[j][m] * dg[m];
        ok = ok && (s > 0.0);
        dg[j] = s;
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            double t = -B[i][j];
#pragma unroll
            for (int m = 0; m < j; ++m) t -= L[i][m] * L[j][m] * dg[m];
            L[i][j] = t / s;
        }
    }
    return ok;
}

// true when M - V B V^T + shift I is positive definite (LDL^T without
// pivoting, in double): the part of M outside span(V) has no eigenvalue
// below -shift (up to the coupling ||M V - V B||, which the caller certified)
template <int K>
__device__ __forceinline__ bool refine_rest_pd(const double* __restrict__ Mg,
                                               const double (&V)[9][K], const double (&B)[K][K],
                                               double shift)
{
    double U[9][K];
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int p = 0; p < K; ++p) {
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j) t = fma(V[r][j], B[j][p], t);
            U[r][p] = t;
        }
    double A[45];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double t = __ldg(Mg + pk(i, j));
#pragma unroll
            for (int p = 0; p < K; ++p) t = fma(-U[i][p], V[j][p], t);
            A[pk(i, j)] = t;
        }
    double Lm[45];
    double dg[9];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        double s = A[pk(j, j)] + shift;
#pragma unroll
        for (int m = 0; m < j; ++m) s -= Lm[pk(j, m)] * Lm[pk(j, m)] * dg[m];
        pd = pd && (s > 0.0);
        dg[j] = s;
        const double inv = 1.0 / s;
#pragma unroll
        for (int i = j + 1; i < 9; ++i) {
            double t = A[pk(i, j)];
#pragma unroll
            for (int m = 0; m < j; ++m) t -= Lm[pk(i, m)] * Lm[pk(j, m)] * dg[m];
            Lm[pk(i, j)] = t * inv;
        }
    }
    return pd;
}

// B <- its part below -tau, sum over eigenvalues l < -tau of l g g^T
// (cyclic Jacobi on the k x k B, rotations skipped at |b_pq| <= thr)
template <int K>
__device__ __forceinline__ void refine_negpart(double (&B)[K][K], double tau, double thr)
{
    double A[K][K], G[K][K];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) {
            A[i][j] = B[i][j];
            G[i][j] = i == j ? 1.0 : 0.0;
        }
#pragma unroll 1
    for (int sw = 0; sw < 10; ++sw) {
        bool any = false;
#pragma unroll
        for (int p = 0; p < K; ++p)
#pragma unroll
            for (int q = p + 1; q < K; ++q) {
                const double apq = A[p][q];
                if (!(fabs(apq) > thr)) continue;
                any = true;
                const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = copysign(1.0, th) / (fabs(th) + sqrt(fma(th, th, 1.0)));
                const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const double arp = A[r][p], arq = A[r][q];
                    A[r][p] = fma(c, arp, -s * arq);
                    A[r][q] = fma(s, arp, c * arq);
                }
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = fma(c, apr, -s * aqr);
                    A[q][r] = fma(s, apr, c * aqr);
                }
                A[p][q] = 0.0;
                A[q][p] = 0.0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const double gp = G[r][p], gq = G[r][q];
                    G[r][p] = fma(c, gp, -s * gq);
                    G[r][q] = fma(s, gp, c * gq);
                }
            }
        if (!any) break;
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < K; ++l)
                s = A[l][l] < -tau ? fma(A[l][l] * G[i][l], G[j][l], s) : s;
            B[i][j] = s;
        }
}

}  // namespace sx
