// sx_elements.cu -- per-element energy, gradient and Hessian kernels
// (the parallel element loop of Algorithm 1: gather, evaluate, project,
// stage for assembly).
//
// Stable Neo-Hookean tet4 (§3.1 Eq. 7, App. B): with F = Ds Dm^-1,
// Ic = |F|^2, J = det F, C = cof F (dJ/dF), the density's first and
// second derivatives are P = a F + b C and
//   d2psi/dF2 = a I9 + gam vec(F)vec(F)^T + lam' vec(C)vec(C)^T + b dC/dF,
// a = mu' Ic/(Ic+1), gam = 2 mu'/(Ic+1)^2, b = lam'(J - alpha). Because F
// is linear in the vertices through the shape-function gradients G_a
// (F = sum_a x_a G_a^T), each 3x3 block of the element Hessian has the
// closed form
//   H_ab = V [ a (G_a.G_b) I3 + gam (F G_a)(F G_b)^T + lam' (C G_a)(C G_b)^T
//              + b S(F (G_a x G_b)) ],   S(w)_ik = eps_ikn w_n,
// so no 9x12 map is formed. The same expression with the Hadamard
// combinations K_c of the G_a gives the 9x9 translation-free Hessian M
// that the PSD projection works on (sx_clamp.cuh).
//
// Hinge bending (§6.3 Eq. 13): Q = c (q q^T kron I3), so
// E = k_b c |sum_a q_a x_a|^2 / 2, g_a = k_b c q_a s, H_ab = k_b c q_a q_b I3
// with s = sum_a q_a x_a; Q is PSD and never projected.
//
// Point-triangle barrier (§6.4 Eq. 15) lives in sx_barrier.cuh.
//
// Precision: SX_FP64 computes everything in double. SX_FP32 forms the
// gathered edge vectors (x_a - x_0) in double, then does the element math
// in float; the projection always runs in double.
#include <cuda_runtime.h>

#include "sx_barrier.cuh"
#include "sx_clamp.cuh"
#include "sx_internal.cuh"

namespace sx {

static constexpr int kElemThreads = 128;

int elements_block_threads() { return kElemThreads; }

template <typename R>
struct Vec3 {
    R x, y, z;
};

// ------------------------------------------------------------------ SNH
template <typename R>
struct SnhCore {
    R G[4][3];   // shape-function gradients (row a)
    R F[9];      // row-major
    R C[9];      // cofactor
    R cI, cF, cC, cS;   // V*a, V*gam, V*lam', V*b
};

template <typename R>
__device__ __forceinline__ void cross3(const R* u, const R* v, R* w)
{
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

// Evaluates, always in double, F = Ds Dm^-1 and the rest-relative energy
// E = V (psi(F) - psi(I)) free of cancellation: with D = F - I,
//   Ic - 3 = |D|^2 + 2 tr D,   J - 1 = tr D + c2(D) + det D
// (c2 = sum of principal 2x2 minors), and since alpha - 1 = 3 mu'/(4 lam'),
//   lam'/2 [(J-alpha)^2 - (1-alpha)^2] = lam'/2 (J-1)^2 - 3/4 mu' (J-1),
//   mu'/2 [ln(Ic+1) - ln 4] = mu'/2 log1p((Ic-3)/4).
// No O(1) quantities are subtracted, so the line search can resolve the
// last Newton decreases. Then, in the element precision R, the gradient
// (12, node-major) and the Hessian coefficients.
template <typename R>
__device__ __forceinline__ double snh_core(const double* xg, const double* Dinv, double Vd,
                                           double mud, double lamd, int level, SnhCore<R>& S,
                                           R* g)
{
    double Ds[3][3];  // Ds[i][k] = x_{k+1,i} - x_{0,i}
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) Ds[i][k] = xg[3 * (k + 1) + i] - xg[i];
    double Fd[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Fd[i * 3 + j] = Ds[i][0] * Dinv[0 * 3 + j] + Ds[i][1] * Dinv[1 * 3 + j] +
                            Ds[i][2] * Dinv[2 * 3 + j];
    double D[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = Fd[k] - ((k % 4 == 0) ? 1.0 : 0.0);
    const double trD = D[0] + D[4] + D[8];
    double Ic3 = 2.0 * trD;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ic3 = fma(D[k], D[k], Ic3);
    const double c2 = (D[0] * D[4] - D[1] * D[3]) + (D[0] * D[8] - D[2] * D[6]) +
                      (D[4] * D[8] - D[5] * D[7]);
    const double detD = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                        D[2] * (D[3] * D[7] - D[4] * D[6]);
    const double Jm1 = trD + c2 + detD;
    double psi = 0.5 * mud * Ic3 - 0.5 * mud * log1p(0.25 * Ic3);
    if (lamd != 0.0) psi += 0.5 * lamd * Jm1 * Jm1 - 0.75 * mud * Jm1;
    const double E = Vd * psi;
    if (level >= 1) {
        const R V = (R)Vd, mu = (R)mud, lam = (R)lamd;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S.G[1][j] = (R)Dinv[0 * 3 + j];
            S.G[2][j] = (R)Dinv[1 * 3 + j];
            S.G[3][j] = (R)Dinv[2 * 3 + j];
            S.G[0][j] = (R)(-(Dinv[0 * 3 + j] + Dinv[1 * 3 + j] + Dinv[2 * 3 + j]));
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) S.F[k] = (R)Fd[k];
        const R* F = S.F;
        // cofactor columns: dJ/dF columns are f1 x f2, f2 x f0, f0 x f1
        {
            R f0[3] = {F[0], F[3], F[6]}, f1[3] = {F[1], F[4], F[7]}, f2[3] = {F[2], F[5], F[8]};
            R c0[3], c1[3], cc2[3];
            cross3(f1, f2, c0);
            cross3(f2, f0, c1);
            cross3(f0, f1, cc2);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                S.C[i * 3 + 0] = c0[i];
                S.C[i * 3 + 1] = c1[i];
                S.C[i * 3 + 2] = cc2[i];
            }
        }
        const R Ic = (R)(3.0 + Ic3);
        const R inv1 = R(1) / (Ic + R(1));
        const R a = mu * Ic * inv1;
        // lam'(J - alpha) = lam'(J - 1) - 3/4 mu'
        const R b = (lamd != 0.0) ? (R)(lamd * Jm1 - 0.75 * mud) : R(0);
        R P[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k] = a * F[k] + b * S.C[k];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                g[3 * n + i] = V * (P[i * 3 + 0] * S.G[n][0] + P[i * 3 + 1] * S.G[n][1] +
                                    P[i * 3 + 2] * S.G[n][2]);
        S.cI = V * a;
        S.cF = V * R(2) * mu * inv1 * inv1;
        S.cC = V * lam;
        S.cS = V * b;
    }
    return E;
}

// one 3x3 block V[ a (Ga.Gb) I + gam uu^T + lam' vv^T + b S(F (Ga x Gb)) ]
template <typename R>
__device__ __forceinline__ void snh_block(const SnhCore<R>& S, const R* Ga, const R* Gb,
                                          const R* ua, const R* ub, const R* va,
                                          const R* vb, bool diag, R* out)
{
    const R gg = Ga[0] * Gb[0] + Ga[1] * Gb[1] + Ga[2] * Gb[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            out[i * 3 + k] = S.cF * ua[i] * ub[k] + S.cC * va[i] * vb[k] +
                             (i == k ? S.cI * gg : R(0));
    if (!diag) {
        R c[3], w[3];
        cross3(Ga, Gb, c);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            w[i] = S.F[i * 3 + 0] * c[0] + S.F[i * 3 + 1] * c[1] + S.F[i * 3 + 2] * c[2];
        // S(w) = [[0, w2, -w1], [-w2, 0, w0], [w1, -w0, 0]]
        out[1] += S.cS * w[2];
        out[2] -= S.cS * w[1];
        out[3] -= S.cS * w[2];
        out[5] += S.cS * w[0];
        out[6] += S.cS * w[1];
        out[7] -= S.cS * w[0];
    }
}

template <typename R>
__device__ __forceinline__ void matvec3(const R* M, const R* v, R* o)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = M[i * 3 + 0] * v[0] + M[i * 3 + 1] * v[1] + M[i * 3 + 2] * v[2];
}

// 9x9 translation-free Hessian M (double, both triangles) of an SNH tet.
template <typename R>
__device__ __forceinline__ void snh_M(const SnhCore<R>& S, double* M)
{
    R K[3][3];   // K_c, c = 1..3 stored at [c-1]
#pragma unroll
    for (int j = 0; j < 3; ++j)
        had_fwd(S.G[0][j], S.G[1][j], S.G[2][j], S.G[3][j], K[0][j], K[1][j], K[2][j]);
    R u[3][3], v[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        matvec3(S.F, K[c], u[c]);
        matvec3(S.C, K[c], v[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = c; d < 3; ++d) {
            R blk[9];
            snh_block(S, K[c], K[d], u[c], u[d], v[c], v[d], c == d, blk);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    M[(3 * c + i) * 9 + (3 * d + k)] = (double)blk[i * 3 + k];
                    M[(3 * d + k) * 9 + (3 * c + i)] = (double)blk[i * 3 + k];
                }
        }
}

// ------------------------------------------------------------------ output
// Writes the 10 upper blocks of H - sum_t lam_t u_t u_t^T, with the blocks
// produced by `blockfn(a, b, out9)` in the element precision.
template <typename R, typename HT, typename BlockFn>
__device__ __forceinline__ void write_blocks(BlockFn blockfn, int nneg, const double* lamv,
                                             const double* U, HT* staged, double* full,
                                             int* nonfinite)
{
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
            R blk[9];
            blockfn(a, b, blk);
            double o[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = (double)blk[k];
            for (int t = 0; t < nneg; ++t) {
                const double* u = U + 12 * t;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        o[i * 3 + k] = fma(-lamv[t] * u[3 * a + i], u[3 * b + k], o[i * 3 + k]);
            }
            bool bad = false;
#pragma unroll
            for (int k = 0; k < 9; ++k) bad |= !isfinite(o[k]);
            if (bad) *nonfinite = 1;
            if (staged) {
                HT* dst = staged + 9 * up_index(a, b);
#pragma unroll
                for (int k = 0; k < 9; ++k) dst[k] = (HT)o[k];
            }
            if (full) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        full[(3 * a + i) * 12 + (3 * b + k)] = o[i * 3 + k];
                        full[(3 * b + k) * 12 + (3 * a + i)] = o[i * 3 + k];
                    }
            }
        }
}

// negative eigenpairs of M mapped to 12-vectors u = (Hd kron I3)(0, v)
__device__ __forceinline__ int project_negatives(double* M, double* lamv, double* U,
                                                 int* failed)
{
    double V9[81];
    double fro;
    int k = neg_eigs9(M, lamv, V9, &fro);
    if (k < 0) {
        *failed = 1;
        return 0;
    }
    for (int t = 0; t < k; ++t) {
        const double* v = V9 + 9 * t;
        double* u = U + 12 * t;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            had_inv(v[i], v[3 + i], v[6 + i], u[i], u[3 + i], u[6 + i], u[9 + i]);
    }
    return k;
}

// ------------------------------------------------------------------ kernel
struct ThreadOut {
    double E;
    int bad;        // barrier d <= 0
    int nonfinite;
    int clamped;
};

template <typename R, typename HT>
__device__ void eval_snh(const ElemLaunch& L, const SceneDev& S, const ElemBlock& B,
                         int64_t e, ThreadOut& o)
{
    const int4 t = B.conn[e];
    double xg[12];
    const int nid[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const double* p = S.x + 3 * (int64_t)nid[a];
        xg[3 * a + 0] = p[0];
        xg[3 * a + 1] = p[1];
        xg[3 * a + 2] = p[2];
    }
    double Dinv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Dinv[k] = B.Dminv[(int64_t)k * B.n + e];
    SnhCore<R> C;
    R g[12];
    o.E = snh_core<R>(xg, Dinv, B.V[e], B.mu[e], B.lam[e], L.level, C, g);
    if (!isfinite(o.E)) o.nonfinite = 1;
    const int64_t gid = B.base + e;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gout[k] = (double)g[k];
            if (!isfinite((double)g[k])) o.nonfinite = 1;
        }
    }
    if (L.level >= 2) {
        double lamv[9];
        double U[12 * 9];
        int nneg = 0;
        if (L.project) {
            double M[81];
            snh_M<R>(C, M);
            int failed = 0;
            nneg = project_negatives(M, lamv, U, &failed);
            if (failed) o.nonfinite = 1;
            o.clamped = nneg > 0;
        }
        R u[4][3], v[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            matvec3(C.F, C.G[a], u[a]);
            matvec3(C.C, C.G[a], v[a]);
        }
        auto blockfn = [&](int a, int b, R* out) {
            snh_block(C, C.G[a], C.G[b], u[a], u[b], v[a], v[b], a == b, out);
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, nneg, lamv, U, staged, full, &o.nonfinite);
    }
}

template <typename R, typename HT>
__device__ void eval_hinge(const ElemLaunch& L, const SceneDev& S, const ElemBlock& B,
                           int64_t e, ThreadOut& o)
{
    const int4 t = B.conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    R q[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] = (R)B.q[(int64_t)a * B.n + e];
    const R kc = (R)(B.kb * B.c[e]);
    // s = sum_a q_a x_a, formed relative to node 0 (sum_a q_a = 0 for a
    // translation-free hinge; the relative form only improves rounding and
    // is exact for any q when the missing q-sum term is added back)
    double x0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) x0[i] = S.x[3 * (int64_t)nid[0] + i];
    double qd[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) qd[a] = B.q[(int64_t)a * B.n + e];
    const double qs = qd[0] + qd[1] + qd[2] + qd[3];
    double sd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) sd[i] = qs * x0[i];
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) sd[i] += qd[a] * (S.x[3 * (int64_t)nid[a] + i] - x0[i]);
    o.E = 0.5 * B.kb * B.c[e] * (sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
    const R s[3] = {(R)sd[0], (R)sd[1], (R)sd[2]};
    if (!isfinite(o.E)) o.nonfinite = 1;
    const int64_t gid = B.base + e;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) gout[3 * a + i] = (double)(kc * q[a] * s[i]);
    }
    if (L.level >= 2) {
        auto blockfn = [&](int a, int b, R* out) {
            R h = kc * q[a] * q[b];
#pragma unroll
            for (int k = 0; k < 9; ++k) out[k] = (k % 4 == 0) ? h : R(0);
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, 0, nullptr, nullptr, staged, full, &o.nonfinite);
    }
}

template <typename R, typename HT>
__device__ void eval_barrier(const ElemLaunch& L, const SceneDev& S, const ElemBlock& B,
                             int64_t e, ThreadOut& o)
{
    const int4 t = B.conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    // coordinates relative to the point, formed in double
    double xr[12];
    double p0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) p0[i] = S.x[3 * (int64_t)nid[0] + i];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) xr[3 * a + i] = S.x[3 * (int64_t)nid[a] + i] - p0[i];
    BarrierOut<R> bo;
    int st = barrier_eval<R>(xr, (R)B.dhat, (R)B.kappa, L.level, bo);
    double Ed = (double)bo.E;
    if (sizeof(R) != sizeof(double)) {
        // the energy (line-search quantity) is always evaluated in double
        BarrierOut<double> bd;
        int sd = barrier_eval<double>(xr, B.dhat, B.kappa, 0, bd);
        if (sd < 0) st = sd;
        Ed = (sd == 1) ? bd.E : 0.0;
        if (sd != 1 && st == 1) st = sd;
    }
    const int64_t gid = B.base + e;
    if (st < 0) o.bad = 1;
    o.E = (st == 1) ? Ed : 0.0;
    if (!isfinite(o.E)) o.nonfinite = 1;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) gout[k] = (st == 1) ? (double)bo.g[k] : 0.0;
    }
    if (L.level >= 2) {
        double lamv[9];
        double U[12 * 9];
        int nneg = 0;
        if (st == 1 && L.project) {
            double M[81];
            // M = (Hd kron I3) H (Hd kron I3) restricted to the modes c, d = 1..3
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    // transform rows: T[a][c] blocks, entry (i,k)
                    R Tm[4][3];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        R h0 = bo.H[(3 * a + i) * 12 + 0 * 3 + k];
                        R h1 = bo.H[(3 * a + i) * 12 + 1 * 3 + k];
                        R h2 = bo.H[(3 * a + i) * 12 + 2 * 3 + k];
                        R h3 = bo.H[(3 * a + i) * 12 + 3 * 3 + k];
                        had_fwd(h0, h1, h2, h3, Tm[a][0], Tm[a][1], Tm[a][2]);
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        R y1, y2, y3;
                        had_fwd(Tm[0][d], Tm[1][d], Tm[2][d], Tm[3][d], y1, y2, y3);
                        M[(0 * 3 + i) * 9 + (3 * d + k)] = (double)y1;
                        M[(1 * 3 + i) * 9 + (3 * d + k)] = (double)y2;
                        M[(2 * 3 + i) * 9 + (3 * d + k)] = (double)y3;
                    }
                }
            // symmetrize exactly
#pragma unroll
            for (int r = 0; r < 9; ++r)
#pragma unroll
                for (int c = r + 1; c < 9; ++c) {
                    double m = 0.5 * (M[r * 9 + c] + M[c * 9 + r]);
                    M[r * 9 + c] = m;
                    M[c * 9 + r] = m;
                }
            int failed = 0;
            nneg = project_negatives(M, lamv, U, &failed);
            if (failed) o.nonfinite = 1;
            o.clamped = nneg > 0;
        }
        auto blockfn = [&](int a, int b, R* out) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    out[i * 3 + k] = (st == 1) ? bo.H[(3 * a + i) * 12 + 3 * b + k] : R(0);
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, nneg, lamv, U, staged, full, &o.nonfinite);
    }
}

template <typename R, typename HT>
__global__ void __launch_bounds__(kElemThreads)
k_elements(ElemLaunch L)
{
    __shared__ double sE[kElemThreads];
    __shared__ int sI[3][kElemThreads];
    __shared__ int tile_id;
    for (;;) {
        if (threadIdx.x == 0) tile_id = atomicAdd(L.queue, 1);
        __syncthreads();
        const int ti = tile_id;
        __syncthreads();
        if (ti >= L.ntiles) return;
        const Tile T = L.tiles[ti];
        const SceneDev& S = L.scenes[T.scene];
        ThreadOut o{0.0, 0, 0, 0};
        if (S.sc == nullptr || S.sc->active) {
            const ElemBlock& B = S.blk[T.blk];
            if ((int)threadIdx.x < T.count) {
                const int64_t e = T.start + threadIdx.x;
                if (B.kind == SX_KIND_SNH_TET4)
                    eval_snh<R, HT>(L, S, B, e, o);
                else if (B.kind == SX_KIND_HINGE4)
                    eval_hinge<R, HT>(L, S, B, e, o);
                else
                    eval_barrier<R, HT>(L, S, B, e, o);
                if (L.out_E) L.out_E[e] = o.E;
                else S.Ee[B.base + e] = o.E;
            }
        }
        // fixed-order tile reductions
        sE[threadIdx.x] = o.E;
        sI[0][threadIdx.x] = o.bad;
        sI[1][threadIdx.x] = o.nonfinite;
        sI[2][threadIdx.x] = o.clamped;
        __syncthreads();
        for (int w = kElemThreads / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) {
                sE[threadIdx.x] += sE[threadIdx.x + w];
                sI[0][threadIdx.x] += sI[0][threadIdx.x + w];
                sI[1][threadIdx.x] += sI[1][threadIdx.x + w];
                sI[2][threadIdx.x] += sI[2][threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (L.tile_E) L.tile_E[ti] = sE[0];
            if (L.tile_bad) L.tile_bad[ti] = sI[0][0];
            if (L.tile_nonfinite) L.tile_nonfinite[ti] = sI[1][0];
            if (L.tile_clamped) L.tile_clamped[ti] = sI[2][0];
        }
        __syncthreads();
    }
}

const void* elements_kernel(int precision)
{
    return precision == SX_FP32 ? (const void*)k_elements<float, float>
                                : (const void*)k_elements<double, double>;
}

cudaError_t launch_elements(const ElemLaunch& L, int grid, cudaStream_t s)
{
    if (L.ntiles == 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(L.queue, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    if (L.precision == SX_FP32)
        k_elements<float, float><<<grid, kElemThreads, 0, s>>>(L);
    else
        k_elements<double, double><<<grid, kElemThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace sx
