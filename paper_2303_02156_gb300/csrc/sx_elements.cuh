// sx_elements.cuh -- per-element energy, gradient and Hessian kernels
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
// Other tet4 densities (§6.1, App. B; compiled into separate
// instantiations, KINDS bit 16): Neo-Hookean, fixed co-rotational and ARAP
// have the same Hessian form with gam = 0 and their own coefficients; St.
// Venant-Kirchhoff has its own blocks (see model_core).
//
// Point-triangle barrier (§6.4 Eq. 15) lives in sx_barrier.cuh; the
// lagged IPC friction (§6.4, KINDS bit 32) is eval_friction and the 10- and
// 20-node tets (§6.2 Eq. 12, KINDS bit 64) are tetho_tile.
//
// Precision: SX_FP64 computes everything in double. SX_FP32 forms the
// gathered edge vectors (x_a - x_0) in double, then does the element math
// in float; the projection always runs in double.
//
// The element kernel k_elements<R, HT, KINDS> is instantiated in four
// translation units (sx_elements.cu: KINDS 1, 7; sx_elements_fproj.cu: 9,
// 15; sx_elements_models.cu: 25, 63; sx_elements_ho.cu: 64, 127) so that
// they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "sx_barrier.cuh"
#include "sx_clamp.cuh"
#include "sx_internal.cuh"

namespace sx {

static constexpr int kElemThreads = 128;
// projection block sizes the launch may use: 32, 64, 128 (the default) or
// 256, picked by sx_autotune; each thread keeps its 9x9 eigenvector matrix
// (648 B) in dynamic shared memory
static constexpr int kClampThreads = 64;
// sharing: unused dynamic shared memory per block that lowers the resident
// blocks per SM by one (from the register limit of 255-register threads):
// 32 threads 20.3 + 8 KB (8 -> 7), 64 threads 40.5 + 17 KB (4 -> 3),
// 128 threads 81 + 32 KB (2 -> 1); 256-thread blocks are alone on an SM
__host__ __device__ constexpr int clamp_share_pad(int nt)
{
    return nt == 32 ? 8 * 1024 : nt == 64 ? 17 * 1024 : nt == 128 ? 32 * 1024 : 0;
}
static constexpr int kClampMaxSmem = 81 * 8 * 256;

template <typename R>
struct Vec3 {
    R x, y, z;
};

// ------------------------------------------------------------------ SNH
template <typename R>
struct SnhCore {
    R G[4][3];   // shape-function gradients (row a)
    R F[9];      // row-major
    R C[9];      // cofactor (the models' and quadrature cores; the SNH tet4 path
                 // takes cof(F) G_a from the deformed edges instead)
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
        const R Ic = (R)(3.0 + Ic3);
        const double Icd = 3.0 + Ic3;
        const double invd = 1.0 / (Icd + 1.0);   // the one division: 1 / (Ic + 1)
        const R inv1 = (R)invd;
        const R a = mu * Ic * inv1;
        // lam'(J - alpha) = lam'(J - 1) - 3/4 mu'
        const R b = (lamd != 0.0) ? (R)(lamd * Jm1 - 0.75 * mud) : R(0);
        // P = a F + b cof F. Its two O(mu') parts cancel at rest, so it is
        // formed from D = F - I: cof(I + D) = I + (tr D) I - D^T + cof D gives
        // P = (a + b) I + a D + b ((tr D) I - D^T + cof D), where
        // a + b = mu' Ic3 / (4 (Ic + 1)) + lam' (J - 1) (alpha = 1 + 3 mu' / (4 lam'))
        // is taken in double; the rest is O(mu' |D|) and keeps R's relative
        // precision (in FP32 this is what lets the assembled forces resolve
        // below float epsilon times mu')
        const R s0 = (lamd != 0.0) ? (R)(0.25 * mud * Ic3 * invd + lamd * Jm1)
                                   : (R)(mud * Icd * invd);
        R Dr[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Dr[k] = (R)D[k];
        const R trr = (R)trD;
        R cofD[9];
        cofD[0] = Dr[4] * Dr[8] - Dr[5] * Dr[7];
        cofD[1] = Dr[5] * Dr[6] - Dr[3] * Dr[8];
        cofD[2] = Dr[3] * Dr[7] - Dr[4] * Dr[6];
        cofD[3] = Dr[2] * Dr[7] - Dr[1] * Dr[8];
        cofD[4] = Dr[0] * Dr[8] - Dr[2] * Dr[6];
        cofD[5] = Dr[1] * Dr[6] - Dr[0] * Dr[7];
        cofD[6] = Dr[1] * Dr[5] - Dr[2] * Dr[4];
        cofD[7] = Dr[2] * Dr[3] - Dr[0] * Dr[5];
        cofD[8] = Dr[0] * Dr[4] - Dr[1] * Dr[3];
        R P[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                P[i * 3 + j] = ((i == j) ? s0 + b * trr : R(0)) + a * Dr[i * 3 + j] +
                               b * (cofD[i * 3 + j] - Dr[j * 3 + i]);
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

// ---- SNH tet4 Hessian blocks from the deformed edges
// With Dm = [X1 - X0, X2 - X0, X3 - X0], G_1..G_3 the rows of Dm^-1 and
// G_0 = -(G_1 + G_2 + G_3), adj(Dm^-1) = Dm^-1^-1 det(Dm^-1) gives
// G_2 x G_3 = (X1 - X0)/det(Dm), G_3 x G_1 = (X2 - X0)/det(Dm),
// G_1 x G_2 = (X3 - X0)/det(Dm); since F (X_k - X0) = x_k - x0 = ds_{k-1},
// the skew vectors of the blocks are scaled deformed edges:
//   F(G_2 x G_3) = ds0 / det(Dm), F(G_1 x G_3) = -ds1 / det(Dm),
//   F(G_1 x G_2) = ds2 / det(Dm), F(G_0 x G_1) = (ds2 - ds1) / det(Dm),
//   F(G_0 x G_2) = (ds0 - ds2) / det(Dm), F(G_0 x G_3) = (ds1 - ds0) / det(Dm),
// and cof(F) G_a = J F^-T G_a (the deformed area vectors over det(Dm)):
//   cof(F) G_1 = ds1 x ds2 / det(Dm), cof(F) G_2 = ds2 x ds0 / det(Dm),
//   cof(F) G_3 = ds0 x ds1 / det(Dm), cof(F) G_0 = -(sum of the three).
// For the Hadamard combinations K_c of the G_a (c = 1..3), F (K_c x K_d) is
// again an edge combination: (ds2 - ds1 - ds0), (ds1 + ds2 - ds0),
// (ds1 - ds2 - ds0) over det(Dm) for (c, d) = (1, 2), (1, 3), (2, 3). This
// takes no cofactor matrix, no F (G_a x G_b) products and no cof(F) G_a
// matvecs; a diagonal block (a = b: no skew part) is formed once per pair
// of its symmetric entries.

__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

// block uSa ub^T + vSa vb^T + cIgg I (+ the skew matrix of ws off the
// diagonal); uSa = V gam u_a, vSa = V lam' v_a, ws = V b w_ab
template <typename R>
__device__ __forceinline__ void snh_block_e(const R* uSa, const R* ub, const R* vSa, const R* vb,
                                            R cIgg, const R* ws, bool diag, R* out)
{
    if (diag) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = i; k < 3; ++k) {
                const R t = fma_r(vSa[i], vb[k], uSa[i] * ub[k]) + (i == k ? cIgg : R(0));
                out[i * 3 + k] = t;
                out[k * 3 + i] = t;
            }
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            out[i * 3 + k] = fma_r(vSa[i], vb[k], uSa[i] * ub[k]) + (i == k ? cIgg : R(0));
    // S(w) = [[0, w2, -w1], [-w2, 0, w0], [w1, -w0, 0]]
    out[1] += ws[2];
    out[2] -= ws[1];
    out[3] -= ws[2];
    out[5] += ws[0];
    out[6] += ws[1];
    out[7] -= ws[0];
}

// V b F (G_a x G_b) for node pair a < b, from the deformed edges ds
// (sw = V b / det(Dm))
template <typename R>
__device__ __forceinline__ void snh_node_skew(int a, int b, const R (&ds)[3][3], R sw, R* ws)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R t;
        if (a == 2) t = ds[0][i];                       // (2, 3)
        else if (a == 1) t = b == 2 ? ds[2][i] : -ds[1][i];   // (1, 2), (1, 3)
        else if (b == 1) t = ds[2][i] - ds[1][i];       // (0, 1)
        else if (b == 2) t = ds[0][i] - ds[2][i];       // (0, 2)
        else t = ds[1][i] - ds[0][i];                   // (0, 3)
        ws[i] = sw * t;
    }
}

// the same for Hadamard mode pair c < d (0-based c, d: modes c + 1, d + 1)
template <typename R>
__device__ __forceinline__ void snh_mode_skew(int c, int d, const R (&ds)[3][3], R sw, R* ws)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R t;
        if (c == 1) t = ds[1][i] - ds[2][i] - ds[0][i];        // (2, 3)
        else if (d == 1) t = ds[2][i] - ds[1][i] - ds[0][i];   // (1, 2)
        else t = ds[1][i] + ds[2][i] - ds[0][i];               // (1, 3)
        ws[i] = sw * t;
    }
}

// u_a = F G_a and v_a = cof(F) G_a (node a = 0..3) from the core and the
// deformed edges (dD = 1 / det(Dm))
template <typename R>
__device__ __forceinline__ void snh_uv(const SnhCore<R>& S, const R (&ds)[3][3], R dD,
                                       R (&u)[4][3], R (&v)[4][3])
{
#pragma unroll
    for (int a = 0; a < 4; ++a) matvec3(S.F, S.G[a], u[a]);
    cross3(ds[1], ds[2], v[1]);
    cross3(ds[2], ds[0], v[2]);
    cross3(ds[0], ds[1], v[3]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        v[1][i] *= dD;
        v[2][i] *= dD;
        v[3][i] *= dD;
        v[0][i] = -(v[1][i] + v[2][i] + v[3][i]);
    }
}

// 9x9 translation-free Hessian M (double, packed lower) of an SNH tet from
// the node vectors: u, v of the modes are Hadamard combinations of the node
// ones, the K_c those of the G_a
template <typename R>
__device__ __forceinline__ void snh_M_e(const SnhCore<R>& S, const R (&u)[4][3],
                                        const R (&v)[4][3], const R (&ds)[3][3], R sw,
                                        double (&M)[45])
{
    R K[3][3], um[3][3], vm[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        had_fwd(S.G[0][j], S.G[1][j], S.G[2][j], S.G[3][j], K[0][j], K[1][j], K[2][j]);
        had_fwd(u[0][j], u[1][j], u[2][j], u[3][j], um[0][j], um[1][j], um[2][j]);
        had_fwd(v[0][j], v[1][j], v[2][j], v[3][j], vm[0][j], vm[1][j], vm[2][j]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R uS[3], vS[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            uS[i] = S.cF * um[c][i];
            vS[i] = S.cC * vm[c][i];
        }
#pragma unroll
        for (int d = c; d < 3; ++d) {
            const R gg = K[c][0] * K[d][0] + K[c][1] * K[d][1] + K[c][2] * K[d][2];
            R ws[3] = {R(0), R(0), R(0)};
            if (c != d) snh_mode_skew(c, d, ds, sw, ws);
            R blk[9];
            snh_block_e(uS, um[d], vS, vm[d], S.cI * gg, ws, c == d, blk);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (3 * d + k <= 3 * c + i || c != d)
                        M[pk(3 * d + k, 3 * c + i)] = to_f64_bits(blk[i * 3 + k]);
        }
    }
}

// ------------------------------------------------------------------ output
// Writes the 10 upper blocks produced by `blockfn(a, b, out9)` (element
// precision) to the staged buffer, or the full 12x12 to `full`.
template <typename R, typename HT, typename BlockFn>
__device__ __forceinline__ void write_blocks(BlockFn blockfn, HT* staged, double* full,
                                             int* nonfinite)
{
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
            R blk[9];
            blockfn(a, b, blk);
            bool bad = false;
#pragma unroll
            for (int k = 0; k < 9; ++k) bad |= nonfinite_bits(blk[k]);
            if (bad) *nonfinite = 1;
            if (staged) {
                HT* dst = staged + 9 * up_index(a, b);
#pragma unroll
                for (int k = 0; k < 9; ++k) dst[k] = (HT)blk[k];
            }
            if (full) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        full[(3 * a + i) * 12 + (3 * b + k)] = (double)blk[i * 3 + k];
                        full[(3 * b + k) * 12 + (3 * a + i)] = (double)blk[i * 3 + k];
                    }
            }
        }
}

// phase 1 of the projection: queue M unless M + tau I is PD
__device__ __forceinline__ bool queue_if_indefinite(const ElemLaunch& L, int scene, int blk,
                                                    int64_t e, const double (&M)[45])
{
    const int cls = psd_class_f32(M);
    if (cls > 0 || (cls == 0 && psd_by_ldlt(M))) return false;
    const int slot = atomicAdd(L.clamp_count, 1);
    if (slot >= L.clamp_cap) return false;   // cannot happen: capacity = stencils
    double* dst = L.clamp_M + 45 * (int64_t)slot;
#pragma unroll
    for (int k = 0; k < 45; ++k) dst[k] = M[k];
    L.clamp_ref[slot] = ClampRef{scene, blk, e};
    return true;
}

// ------------------------------------------------------------------ kernel
struct ThreadOut {
    double E;
    int bad;        // barrier d <= 0
    int nonfinite;
    int clamped;    // queued for the projection
};

// ---------------------------------------------------------------- F-space projection
// Cyclic Jacobi on a symmetric 3x3 in double (A packed lower: 00,10,11,20,21,22),
// eigenvectors accumulated into the columns of Q (row-major). Stops once
// the off-diagonal is below 1e-17 of the diagonal scale (at most 8 sweeps).
__device__ __forceinline__ void jacobi3(double (&A)[6], double (&Q)[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sw = 0; sw < 8; ++sw) {
        const double off = fabs(A[1]) + fabs(A[3]) + fabs(A[4]);
        const double dia = fabs(A[0]) + fabs(A[2]) + fabs(A[5]);
        if (!(off > 1e-17 * dia)) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const int ipq = pk(p, q), ipp = pk(p, p), iqq = pk(q, q);
            const double apq = A[ipq];
            if (apq == 0.0) continue;
            const double tau = (A[iqq] - A[ipp]) / (2.0 * apq);
            const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
            const double c = rsqrt(fma(t, t, 1.0)), sn = t * c;
            A[ipp] -= t * apq;
            A[iqq] += t * apq;
            A[ipq] = 0.0;
            const int r = 3 - p - q;
            const double arp = A[pk(r, p)], arq = A[pk(r, q)];
            A[pk(r, p)] = c * arp - sn * arq;
            A[pk(r, q)] = sn * arp + c * arq;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double xp = Q[3 * i + p], xq = Q[3 * i + q];
                Q[3 * i + p] = c * xp - sn * xq;
                Q[3 * i + q] = sn * xp + c * xq;
            }
        }
    }
}

// Negative modes of the SNH material Hessian d2psi/dF2 at F. In the frame
// of the signed SVD F = U diag(s) V^T (U, V rotations) the material Hessian
// a I + gam F F^T + lam' C C^T + b dC/dF splits into three twist/flip pairs,
// eigenvalue a - b s_k on (u_i v_j^T + u_j v_i^T)/sqrt2 and a + b s_k on
// (u_i v_j^T - u_j v_i^T)/sqrt2 ({i, j, k} = {0, 1, 2}), and the stretch
// block a I + gam s s^T + lam' p p^T + b K on U diag(q) V^T, with
// p = (s1 s2, s0 s2, s0 s1) and K the symmetric 3x3 with zero diagonal and
// K01 = s2, K02 = s1, K12 = s0. Writes each negative eigenvalue and its unit
// F-space eigenvector as a 3x3 matrix M (row-major); returns their count.
// A mode changes the Hessian block (a, b) of an element by
// -V lambda (M G_a)(M G_b)^T.
__device__ __forceinline__ int snh_neg_modes(const double (&F)[9], double mud, double lamd,
                                             double (&lam)[9], double (&M)[9][9])
{
    double Ic = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ic = fma(F[k], F[k], Ic);
    const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                     F[2] * (F[3] * F[7] - F[4] * F[6]);
    const double a = mud * Ic / (Ic + 1.0);
    const double gam = 2.0 * mud / ((Ic + 1.0) * (Ic + 1.0));
    const double b = (lamd != 0.0) ? lamd * (J - 1.0) - 0.75 * mud : 0.0;
    // V: eigenvectors of F^T F
    double S[6];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q <= p; ++q)
            S[pk(p, q)] = F[p] * F[q] + F[3 + p] * F[3 + q] + F[6 + p] * F[6 + q];
    double Vm[9];
    jacobi3(S, Vm);
    // a proper rotation V
    const double dv = Vm[0] * (Vm[4] * Vm[8] - Vm[5] * Vm[7]) -
                      Vm[1] * (Vm[3] * Vm[8] - Vm[5] * Vm[6]) +
                      Vm[2] * (Vm[3] * Vm[7] - Vm[4] * Vm[6]);
    if (dv < 0.0) {
        Vm[2] = -Vm[2];
        Vm[5] = -Vm[5];
        Vm[8] = -Vm[8];
    }
    // U from F V: the two larger directions by normalization, the third by
    // the right-handed cross product; its singular value keeps the sign of J
    int m = 0;
    if (S[pk(1, 1)] < S[pk(m, m)]) m = 1;
    if (S[pk(2, 2)] < S[pk(m, m)]) m = 2;
    const int i0 = (m + 1) % 3, j0 = (m + 2) % 3;
    double fv[3][3];   // fv[k] = F v_k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
            fv[k][r] = F[3 * r] * Vm[k] + F[3 * r + 1] * Vm[3 + k] + F[3 * r + 2] * Vm[6 + k];
    double U[3][3];   // U[k] = u_k
    double sg[3];
    {
        double fi[3], fj[3], fm[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            fi[r] = (i0 == 0) ? fv[0][r] : (i0 == 1) ? fv[1][r] : fv[2][r];
            fj[r] = (j0 == 0) ? fv[0][r] : (j0 == 1) ? fv[1][r] : fv[2][r];
            fm[r] = (m == 0) ? fv[0][r] : (m == 1) ? fv[1][r] : fv[2][r];
        }
        const double si = sqrt(fi[0] * fi[0] + fi[1] * fi[1] + fi[2] * fi[2]);
        double ui[3], uj[3], um[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) ui[r] = fi[r] / si;
        const double pr = ui[0] * fj[0] + ui[1] * fj[1] + ui[2] * fj[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) uj[r] = fj[r] - pr * ui[r];
        const double nj = sqrt(uj[0] * uj[0] + uj[1] * uj[1] + uj[2] * uj[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) uj[r] /= nj;
        const double sj = uj[0] * fj[0] + uj[1] * fj[1] + uj[2] * fj[2];
        cross3(ui, uj, um);
        const double sm = um[0] * fm[0] + um[1] * fm[1] + um[2] * fm[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int r = 0; r < 3; ++r) U[k][r] = (k == i0) ? ui[r] : (k == j0) ? uj[r] : um[r];
            sg[k] = (k == i0) ? si : (k == j0) ? sj : sm;
        }
    }
    int cnt = 0;
    const double h = 0.70710678118654752440;   // 1/sqrt(2)
    // twist / flip pairs: M = (u_i v_j^T +- u_j v_i^T)/sqrt2
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
#pragma unroll
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            const double lambda = a + sgn * b * sg[k];   // sgn -1: symmetric, +1: antisymmetric
            if (!(lambda < 0.0)) continue;
            const double sym = (sgn < 0) ? 1.0 : -1.0;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    M[cnt][3 * r + c] = h * (U[i][r] * Vm[3 * c + j] + sym * U[j][r] * Vm[3 * c + i]);
            lam[cnt++] = lambda;
        }
    }
    // stretch block: M = sum_k Q3[k][e] u_k v_k^T
    const double pv[3] = {sg[1] * sg[2], sg[0] * sg[2], sg[0] * sg[1]};
    double A3[6];
    A3[pk(0, 0)] = a + gam * sg[0] * sg[0] + lamd * pv[0] * pv[0];
    A3[pk(1, 1)] = a + gam * sg[1] * sg[1] + lamd * pv[1] * pv[1];
    A3[pk(2, 2)] = a + gam * sg[2] * sg[2] + lamd * pv[2] * pv[2];
    A3[pk(1, 0)] = gam * sg[1] * sg[0] + lamd * pv[1] * pv[0] + b * sg[2];
    A3[pk(2, 0)] = gam * sg[2] * sg[0] + lamd * pv[2] * pv[0] + b * sg[1];
    A3[pk(2, 1)] = gam * sg[2] * sg[1] + lamd * pv[2] * pv[1] + b * sg[0];
    double Q3[9];
    jacobi3(A3, Q3);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const double lambda = A3[pk(e, e)];
        if (!(lambda < 0.0)) continue;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                M[cnt][3 * r + c] = Q3[0 + e] * U[0][r] * Vm[3 * c + 0] +
                                    Q3[3 + e] * U[1][r] * Vm[3 * c + 1] +
                                    Q3[6 + e] * U[2][r] * Vm[3 * c + 2];
        lam[cnt++] = lambda;
    }
    return cnt;
}

// the same as an out-of-line call, for callers with many live registers
static __device__ __noinline__ int snh_neg_modes_call(const double (&F)[9], double mud, double lamd,
                                               double (&lam)[9], double (&M)[9][9])
{
    return snh_neg_modes(F, mud, lamd, lam, M);
}

// project mode 2 for one SNH tet: removes from its Hessian blocks the
// negative modes of d2psi/dF2 (H = V B^T proj(d2psi/dF2) B). Returns the
// number of modes removed.
template <typename HT>
__device__ int snh_fproj(const double* xg, const double* Dinv, double Vd, double mud,
                         double lamd, HT* staged, double* full)
{
    double F[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double d1 = xg[3 + i] - xg[i], d2 = xg[6 + i] - xg[i], d3 = xg[9 + i] - xg[i];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            F[3 * i + j] = d1 * Dinv[j] + d2 * Dinv[3 + j] + d3 * Dinv[6 + j];
    }
    double lam[9], M[9][9];
    const int cnt = snh_neg_modes(F, mud, lamd, lam, M);
    if (!cnt) return 0;
    double G[4][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        G[1][j] = Dinv[j];
        G[2][j] = Dinv[3 + j];
        G[3][j] = Dinv[6 + j];
        G[0][j] = -(Dinv[j] + Dinv[3 + j] + Dinv[6 + j]);
    }
    for (int md = 0; md < cnt; ++md) {
        double w[12];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int r = 0; r < 3; ++r)
                w[3 * n + r] = M[md][3 * r] * G[n][0] + M[md][3 * r + 1] * G[n][1] +
                               M[md][3 * r + 2] * G[n][2];
        const double sc = Vd * lam[md];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bb = a; bb < 4; ++bb)
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const double wr = sc * w[3 * a + r], wc = w[3 * bb + c];
                        if (staged) {
                            HT* p = staged + 9 * up_index(a, bb) + 3 * r + c;
                            *p = (HT)fma(-wr, wc, (double)*p);
                        } else {
                            double* p = full + (3 * a + r) * 12 + 3 * bb + c;
                            *p = fma(-wr, wc, *p);
                            if (a != bb) {
                                double* q = full + (3 * bb + c) * 12 + 3 * a + r;
                                *q = fma(-wr, wc, *q);
                            }
                        }
                    }
    }
    return cnt;
}

template <typename R, typename HT, bool FPROJ>
__device__ void eval_snh(const ElemLaunch& L, int scene, int blk, const SceneDev& S,
                         const ElemBlock& B, int64_t e, ThreadOut& o)
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
    if (nonfinite_bits(o.E)) o.nonfinite = 1;
    const int64_t gid = B.base + e;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gout[k] = to_f64_bits(g[k]);
            if (nonfinite_bits(g[k])) o.nonfinite = 1;
        }
    }
    if (L.level >= 2) {
        // deformed edges and 1 / det(Dm) (the edge identities above snh_block_e)
        R ds[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) ds[k][i] = (R)(xg[3 * (k + 1) + i] - xg[i]);
        const R dD = (R)(Dinv[0] * (Dinv[4] * Dinv[8] - Dinv[5] * Dinv[7]) -
                         Dinv[1] * (Dinv[3] * Dinv[8] - Dinv[5] * Dinv[6]) +
                         Dinv[2] * (Dinv[3] * Dinv[7] - Dinv[4] * Dinv[6]));
        const R sw = C.cS * dD;
        R u[4][3], v[4][3];
        snh_uv(C, ds, dD, u, v);
        {
            auto blockfn = [&](int a, int b, R* out) {
                R uS[3], vS[3], ws[3] = {R(0), R(0), R(0)};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    uS[i] = C.cF * u[a][i];
                    vS[i] = C.cC * v[a][i];
                }
                if (a != b) snh_node_skew(a, b, ds, sw, ws);
                const R gg = C.G[a][0] * C.G[b][0] + C.G[a][1] * C.G[b][1] + C.G[a][2] * C.G[b][2];
                snh_block_e(uS, u[b], vS, v[b], C.cI * gg, ws, a == b, out);
            };
            HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
            double* full = L.out_H ? L.out_H + 144 * e : nullptr;
            write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
        }
        if (FPROJ && L.project == 2) {
            HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
            double* full = L.out_H ? L.out_H + 144 * e : nullptr;
            o.clamped = snh_fproj<HT>(xg, Dinv, B.V[e], B.mu[e], B.lam[e], staged, full) > 0;
        } else if (L.project) {
            double M[45];
            snh_M_e<R>(C, u, v, ds, sw, M);
            o.clamped = queue_if_indefinite(L, scene, blk, e, M);
        }
    }
}

// ------------------------------------------------------------------ other tet4 densities
// With F = I + D (D formed from the gathered edge vectors in double), the
// energies are written without subtracting O(1) quantities:
//   NH    mu/2 |D|^2 - mu (c2(D) + det D) + mu (u - ln(1+u)) + lambda/2 ln^2(1+u),
//         u = J - 1 = tr D + c2(D) + det D (the same function as
//         mu/2 (Ic - 3) - mu ln J + lambda/2 ln^2 J);
//   StVK  mu |E|^2 + lambda/2 tr(E)^2 with E = (D + D^T + D^T D)/2;
//   COROT k mu |F - R|^2 + lambda/2 u^2, k = 1 (ARAP: k = 1/2).
// Derivatives (R lagged, constant):
//   NH      P = mu F + h C, h = (lambda ln J - mu)/J;
//           d2psi/dF2 = mu I + h' c c^T + h dC/dF, h' = (lambda + mu - lambda ln J)/J^2
//   COROT   P = 2k mu (F - R) + lambda u C;
//           d2psi/dF2 = 2k mu I + lambda c c^T + lambda u dC/dF
//   StVK    P = F S, S = 2 mu E + lambda tr(E) I; with u_a = F G_a
//           H_ab = V [ (G_a.S G_b) I3 + mu (G_a.G_b) F F^T + mu u_b u_a^T + lambda u_a u_b^T ]
// The first two are SNH-shaped (snh_block with gam = 0).
template <typename R>
struct StvkCore {
    R Sm[9];   // V S
    R FF[9];   // V mu F F^T
    R cU, cL;  // V mu, V lambda
};

// u - ln(1 + u): for |u| < 1/16 the series u^2 sum_{j=0}^{18} (-1)^j u^j / (j + 2)
// in Horner form (the tail beyond is below 1e-20 of the value), the
// direct difference otherwise.
__device__ __forceinline__ double u_minus_log1p(double u)
{
    if (fabs(u) < 0.0625) {
        double t = 1.0 / 20.0;
#pragma unroll
        for (int j = 17; j >= 0; --j) t = fma(t, u, ((j & 1) ? -1.0 : 1.0) / (double)(j + 2));
        return u * u * t;
    }
    return u - log1p(u);
}

// E (double) of one tet of model != SNH; at level >= 1 the gradient g (R)
// and the Hessian coefficients (S for the SNH-shaped models, T for StVK).
// Sets bad for an invalid state (NH with J <= 0).
template <typename R>
__device__ __forceinline__ double model_core(int model, const double* xg, const double* Dinv,
                                             const double* Rl, double Vd, double mud,
                                             double lamd, int level, SnhCore<R>& S,
                                             StvkCore<R>& T, R* g, int& bad)
{
    double Fd[9], D[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double f = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) f = fma(xg[3 * (k + 1) + i] - xg[i], Dinv[k * 3 + j], f);
            Fd[i * 3 + j] = f;
            D[i * 3 + j] = f - (i == j ? 1.0 : 0.0);
        }
    const double trD = D[0] + D[4] + D[8];
    const double c2 = (D[0] * D[4] - D[1] * D[3]) + (D[0] * D[8] - D[2] * D[6]) +
                      (D[4] * D[8] - D[5] * D[7]);
    const double detD = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                        D[2] * (D[3] * D[7] - D[4] * D[6]);
    const double Jm1 = trD + c2 + detD;
    const double J = 1.0 + Jm1;
    double psi, Pd[9];
    double Eg[9];   // StVK Green strain
    double lnJ = 0.0;
    const double kmu = (model == SX_MODEL_ARAP) ? 0.5 * mud : mud;
    if (model == SX_MODEL_NH) {
        if (!(Jm1 > -1.0)) {
            bad = 1;
            return 0.0;
        }
        double D2 = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) D2 = fma(D[k], D[k], D2);
        lnJ = log1p(Jm1);
        psi = 0.5 * mud * D2 - mud * (c2 + detD) + mud * u_minus_log1p(Jm1) +
              0.5 * lamd * lnJ * lnJ;
    } else if (model == SX_MODEL_STVK) {
        double e2 = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double v = D[i * 3 + j] + D[j * 3 + i];
#pragma unroll
                for (int m = 0; m < 3; ++m) v = fma(D[m * 3 + i], D[m * 3 + j], v);
                Eg[i * 3 + j] = 0.5 * v;
                e2 = fma(Eg[i * 3 + j], Eg[i * 3 + j], e2);
            }
        const double trE = Eg[0] + Eg[4] + Eg[8];
        psi = mud * e2 + 0.5 * lamd * trE * trE;
    } else {   // COROT, ARAP
        double r2 = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double d = Fd[k] - Rl[k];
            Pd[k] = d;
            r2 = fma(d, d, r2);
        }
        psi = kmu * r2 + 0.5 * lamd * Jm1 * Jm1;
    }
    const double E = Vd * psi;
    if (level < 1) return E;
    const R V = (R)Vd;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        S.G[1][j] = (R)Dinv[0 * 3 + j];
        S.G[2][j] = (R)Dinv[1 * 3 + j];
        S.G[3][j] = (R)Dinv[2 * 3 + j];
        S.G[0][j] = (R)(-(Dinv[0 * 3 + j] + Dinv[1 * 3 + j] + Dinv[2 * 3 + j]));
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) S.F[k] = (R)Fd[k];
    R P[9];
    if (model == SX_MODEL_STVK) {
        const double trE = Eg[0] + Eg[4] + Eg[8];
        R Sr[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Sr[k] = (R)(2.0 * mud * Eg[k] + ((k % 4 == 0) ? lamd * trE : 0.0));
            T.Sm[k] = V * Sr[k];
        }
        // P = F S = S + D S (S is O(|D|): keeps R's relative precision)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                P[i * 3 + j] = Sr[i * 3 + j] + (R)D[i * 3 + 0] * Sr[0 * 3 + j] +
                               (R)D[i * 3 + 1] * Sr[1 * 3 + j] + (R)D[i * 3 + 2] * Sr[2 * 3 + j];
        const R mu = (R)mud;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                T.FF[i * 3 + k] = V * mu * (S.F[i * 3 + 0] * S.F[k * 3 + 0] +
                                            S.F[i * 3 + 1] * S.F[k * 3 + 1] +
                                            S.F[i * 3 + 2] * S.F[k * 3 + 2]);
        T.cU = V * mu;
        T.cL = V * (R)lamd;
    } else {
        const R* F = S.F;
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
        S.cF = R(0);
        if (model == SX_MODEL_NH) {
            // P = (mu + h) I + mu D + h ((tr D) I - D^T + cof D) (cof(I + D) =
            // (1 + tr D) I - D^T + cof D), mu + h = (mu u + lambda ln J)/J in
            // double: the O(mu) parts of mu F and h C cancel at rest
            const double h = (lamd * lnJ - mud) / J;
            const double s0 = (mud * Jm1 + lamd * lnJ) / J;
            R cofD[9];
            cofD[0] = (R)(D[4] * D[8] - D[5] * D[7]);
            cofD[1] = (R)(D[5] * D[6] - D[3] * D[8]);
            cofD[2] = (R)(D[3] * D[7] - D[4] * D[6]);
            cofD[3] = (R)(D[2] * D[7] - D[1] * D[8]);
            cofD[4] = (R)(D[0] * D[8] - D[2] * D[6]);
            cofD[5] = (R)(D[1] * D[6] - D[0] * D[7]);
            cofD[6] = (R)(D[1] * D[5] - D[2] * D[4]);
            cofD[7] = (R)(D[2] * D[3] - D[0] * D[5]);
            cofD[8] = (R)(D[0] * D[4] - D[1] * D[3]);
            const R hr = (R)h, mr = (R)mud, sr = (R)s0, tr = (R)trD;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    P[i * 3 + j] = ((i == j) ? sr + hr * tr : R(0)) + mr * (R)D[i * 3 + j] +
                                   hr * (cofD[i * 3 + j] - (R)D[j * 3 + i]);
            S.cI = V * mr;
            S.cC = V * (R)((lamd + mud - lamd * lnJ) / (J * J));
            S.cS = V * hr;
        } else {
            const R k2 = (R)(2.0 * kmu), lr = (R)lamd, ur = (R)Jm1;
#pragma unroll
            for (int k = 0; k < 9; ++k) P[k] = k2 * (R)Pd[k] + lr * ur * S.C[k];
            S.cI = V * k2;
            S.cC = V * lr;
            S.cS = V * lr * ur;
        }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            g[3 * n + i] = V * (P[i * 3 + 0] * S.G[n][0] + P[i * 3 + 1] * S.G[n][1] +
                                P[i * 3 + 2] * S.G[n][2]);
    return E;
}

// one 3x3 StVK block (a, b) from u_a = F G_a
template <typename R>
__device__ __forceinline__ void stvk_block(const StvkCore<R>& T, const R* Ga, const R* Gb,
                                           const R* ua, const R* ub, R* out)
{
    R sg[3];
    matvec3(T.Sm, Gb, sg);
    const R gsg = Ga[0] * sg[0] + Ga[1] * sg[1] + Ga[2] * sg[2];
    const R gg = Ga[0] * Gb[0] + Ga[1] * Gb[1] + Ga[2] * Gb[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            out[i * 3 + k] = gg * T.FF[i * 3 + k] + T.cU * ub[i] * ua[k] +
                             T.cL * ua[i] * ub[k] + (i == k ? gsg : R(0));
}

template <typename R, typename HT>
__device__ __noinline__ void eval_model(const ElemLaunch& L, int scene, int blk, const SceneDev& S,
                           const ElemBlock& B, int64_t e, ThreadOut& o)
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
    double Dinv[9], Rl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Dinv[k] = B.Dminv[(int64_t)k * B.n + e];
    const int model = B.model;
    const bool lagged = model == SX_MODEL_COROT || model == SX_MODEL_ARAP;
#pragma unroll
    for (int k = 0; k < 9; ++k) Rl[k] = lagged ? B.R[(int64_t)k * B.n + e] : 0.0;
    SnhCore<R> C;
    StvkCore<R> T;
    R g[12];
    int bad = 0;
    o.E = model_core<R>(model, xg, Dinv, Rl, B.V[e], B.mu[e], B.lam[e], L.level, C, T, g, bad);
    if (bad) o.bad = 1;
    if (nonfinite_bits(o.E)) o.nonfinite = 1;
    const int64_t gid = B.base + e;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gout[k] = bad ? 0.0 : (double)g[k];
            if (!bad && nonfinite_bits(g[k])) o.nonfinite = 1;
        }
    }
    if (L.level >= 2) {
        const bool stvk = model == SX_MODEL_STVK;
        R u[4][3], v[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            matvec3(C.F, C.G[a], u[a]);
            if (!stvk) matvec3(C.C, C.G[a], v[a]);
        }
        auto blockfn = [&](int a, int b, R* out) {
            if (bad) {
#pragma unroll
                for (int k = 0; k < 9; ++k) out[k] = R(0);
            } else if (stvk) {
                stvk_block(T, C.G[a], C.G[b], u[a], u[b], out);
            } else {
                snh_block(C, C.G[a], C.G[b], u[a], u[b], v[a], v[b], a == b, out);
            }
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
        if (L.project && !bad) {
            // 9x9 translation-free block: the same block forms on the
            // Hadamard combinations K_c of the G_a
            R K[3][3], uk[3][3], vk[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
                had_fwd(C.G[0][j], C.G[1][j], C.G[2][j], C.G[3][j], K[0][j], K[1][j], K[2][j]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                matvec3(C.F, K[c], uk[c]);
                if (!stvk) matvec3(C.C, K[c], vk[c]);
            }
            double M[45];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = c; d < 3; ++d) {
                    R bl[9];
                    if (stvk) stvk_block(T, K[c], K[d], uk[c], uk[d], bl);
                    else snh_block(C, K[c], K[d], uk[c], uk[d], vk[c], vk[d], c == d, bl);
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            if (3 * d + k <= 3 * c + i || c != d)
                                M[pk(3 * d + k, 3 * c + i)] = to_f64_bits(bl[i * 3 + k]);
                }
            o.clamped = queue_if_indefinite(L, scene, blk, e, M);
        }
    }
}

// ------------------------------------------------------------------ friction
// Lagged IPC friction (§6.4 friction potential). The lag of a pair holds
// beta (closest-point weights), T (tangent basis, 2 rows), fn and dx_lag.
// With w = dx - dx_lag (dx = p - sum beta_i t_i, formed relative to p),
// u = T w, s = |u|, y = s / dt and k = mu fn:
//   E = k f0(s), f0(s) = dt f(y);  g_u = k (f0'/s) u;
//   H_u = k [ (f0'/s) I2 + ((f0'' - f0'/s) / s^2) u u^T ] with
//   stick (y <= yh): f0'/s = (2/yh - y/yh^2)/dt, (f0'' - f0'/s)/s^2 = -1/(s yh^2 dt^2)
//                    (a term that vanishes with s: 0 at s = 0)
//   slide:           f0'/s = 1/s,               (f0'' - f0'/s)/s^2 = -1/s^3.
// With c = (1, -beta0, -beta1, -beta2): g_a = c_a T^T g_u and
// H_ab = c_a c_b T^T H_u T. H_u is PSD in both regimes: never projected.
template <typename R, typename HT>
__device__ __noinline__ void eval_friction(const ElemLaunch& L, const SceneDev& S,
                                           const ElemBlock& B, int64_t e, ThreadOut& o)
{
    const int4 t = B.conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    const int64_t n = B.n;
    double lag[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) lag[k] = B.flag[(int64_t)k * n + e];
    const double kf = B.mu_f * lag[9];
    double p0[3], w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p0[i] = S.x[3 * (int64_t)nid[0] + i];
        w[i] = -lag[10 + i];
    }
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i] -= lag[a - 1] * (S.x[3 * (int64_t)nid[a] + i] - p0[i]);
    const double u0 = lag[3] * w[0] + lag[4] * w[1] + lag[5] * w[2];
    const double u1 = lag[6] * w[0] + lag[7] * w[1] + lag[8] * w[2];
    const double s = sqrt(u0 * u0 + u1 * u1);
    const double dt = B.dt_f, yh = B.yhat, y = s / dt;
    double f0, a1, a2;
    if (y <= yh) {
        f0 = dt * (y * y * (1.0 / yh - y / (3.0 * yh * yh)) + yh / 3.0);
        a1 = (2.0 / yh - y / (yh * yh)) / dt;
        a2 = s > 0.0 ? -1.0 / (s * yh * yh * dt * dt) : 0.0;
    } else {
        f0 = s;
        a1 = 1.0 / s;
        a2 = -1.0 / (s * s * s);
    }
    o.E = kf * f0;
    if (nonfinite_bits(o.E)) o.nonfinite = 1;
    const int64_t gid = B.base + e;
    const R c[4] = {R(1), (R)(-lag[0]), (R)(-lag[1]), (R)(-lag[2])};
    R T[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int i = 0; i < 3; ++i) T[r][i] = (R)lag[3 + 3 * r + i];
    if (L.level >= 1) {
        const R gu0 = (R)(kf * a1 * u0), gu1 = (R)(kf * a1 * u1);
        R G3[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) G3[i] = T[0][i] * gu0 + T[1][i] * gu1;
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                gout[3 * a + i] = (double)(c[a] * G3[i]);
                if (nonfinite_bits(gout[3 * a + i])) o.nonfinite = 1;
            }
    }
    if (L.level >= 2) {
        const R h00 = (R)(kf * (a1 + a2 * u0 * u0)), h11 = (R)(kf * (a1 + a2 * u1 * u1));
        const R h01 = (R)(kf * a2 * u0 * u1);
        R M3[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                M3[i * 3 + j] = T[0][i] * (h00 * T[0][j] + h01 * T[1][j]) +
                                T[1][i] * (h01 * T[0][j] + h11 * T[1][j]);
        auto blockfn = [&](int a, int b, R* out) {
            const R cc = c[a] * c[b];
#pragma unroll
            for (int k = 0; k < 9; ++k) out[k] = cc * M3[k];
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
    }
}

// ------------------------------------------------------------------ high-order tets
// psi(F) (double, rest-relative, cancellation-free as for the linear tet)
// and, at level >= 1, P and the Hessian coefficients of SNH at one point
// with unit volume (the caller scales by w det J0).
template <typename R>
__device__ __forceinline__ double snh_point(const double (&Fd)[9], double mud, double lamd,
                                            int level, SnhCore<R>& S, R (&P)[9])
{
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
    if (level < 1) return psi;
#pragma unroll
    for (int k = 0; k < 9; ++k) S.F[k] = (R)Fd[k];
    {
        const R* F = S.F;
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
    const double Icd = 3.0 + Ic3;
    const R inv1 = (R)(1.0 / (Icd + 1.0));
    const R a = (R)(mud * Icd / (Icd + 1.0));
    const R b = (lamd != 0.0) ? (R)(lamd * Jm1 - 0.75 * mud) : R(0);
    const R s0 = (lamd != 0.0) ? (R)(mud * Ic3 / (4.0 * (Icd + 1.0)) + lamd * Jm1)
                               : (R)(mud * Icd / (Icd + 1.0));
    R Dr[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Dr[k] = (R)D[k];
    const R trr = (R)trD;
    R cofD[9];
    cofD[0] = Dr[4] * Dr[8] - Dr[5] * Dr[7];
    cofD[1] = Dr[5] * Dr[6] - Dr[3] * Dr[8];
    cofD[2] = Dr[3] * Dr[7] - Dr[4] * Dr[6];
    cofD[3] = Dr[2] * Dr[7] - Dr[1] * Dr[8];
    cofD[4] = Dr[0] * Dr[8] - Dr[2] * Dr[6];
    cofD[5] = Dr[1] * Dr[6] - Dr[0] * Dr[7];
    cofD[6] = Dr[1] * Dr[5] - Dr[2] * Dr[4];
    cofD[7] = Dr[2] * Dr[3] - Dr[0] * Dr[5];
    cofD[8] = Dr[0] * Dr[4] - Dr[1] * Dr[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i * 3 + j] = ((i == j) ? s0 + b * trr : R(0)) + a * Dr[i * 3 + j] +
                           b * (cofD[i * 3 + j] - Dr[j * 3 + i]);
    S.cI = a;
    S.cF = R(2) * (R)mud * inv1 * inv1;
    S.cC = (R)lamd;
    S.cS = b;
    return psi;
}

// 10- and 20-node tets (§6.2 Eq. 12): E = sum_q wd_q psi(F_q) with
// wd_q = w_q det J0_q, F_q = sum_a x_a G_qa^T and G_qa = J0_q^-T dN_a(xi_q).
// Each point adds SNH blocks of the linear tet's form with V -> wd_q and
// G_a -> G_qa; with projection the negative modes of d2psi/dF2 at F_q are
// removed from them (the per-point F-space projection). For the fixed
// pattern an element is S four-node sub-stencils covering its node pairs:
// each Hessian block (a, b) belongs to the sub-stencil that owns the pair,
// each node gradient to the one that owns the node, the energy to the
// first; the other slots of the sub-stencils hold zeros. Two launches
// before the element kernel:
//   k_tetho_points, one thread per (element, point): F_q from all K
//     nodes, psi, P and the Hessian coefficients into the element's record
//     (ho_rec, [element][point][kHoRec]), the negative modes (with
//     projection) into ho_modes;
//   k_tetho_blocks, one element per group of threads: the element's records
//     and modes into shared memory, then G_qa, F G_qa and cof(F) G_qa for
//     every (point, node), then one thread per owned block (a, b) summing
//     its SNH block over the points (nine accumulators, no thread handles
//     more than one block, nothing is recomputed per sub-stencil), one per
//     node gradient, and the zeros of the unowned slots.
// The element kernel's tiles of these blocks then only sum the staged
// energies and the non-finite flags (tetho_tile).
template <typename R>
__device__ __forceinline__ void tetho_point(const ElemLaunch& L, const SceneDev& S,
                                            const ElemBlock& B, int64_t e, int q)
{
    const int K = B.ho_K, nq = B.ho_nq;
    const int64_t ne = B.ho_n;
    const bool proj = L.level >= 2 && L.project;
    const double mud = B.mu[e], lamd = B.lam[e];
    double* r = B.ho_rec + (e * nq + q) * kHoRec;
    double Ji[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Ji[k] = B.ho_Jinv[((int64_t)q * 9 + k) * ne + e];
    const double wd = B.ho_wdet[(int64_t)q * ne + e];
    // Ds = sum_a (x_a - x_0) dN_a^T, F = Ds J0^-1
    const double* x0 = S.x + 3 * (int64_t)B.ho_conn[e];
    const double* dq = B.ho_dN + q * K * 3;
    double Ds[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 1; a < K; ++a) {
        const double* p = S.x + 3 * (int64_t)B.ho_conn[(int64_t)a * ne + e];
        const double* dn = dq + 3 * a;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double xi = p[i] - x0[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) Ds[3 * i + c] = fma(xi, dn[c], Ds[3 * i + c]);
        }
    }
    double Fd[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Fd[3 * i + c] = Ds[3 * i] * Ji[c] + Ds[3 * i + 1] * Ji[3 + c] + Ds[3 * i + 2] * Ji[6 + c];
    SnhCore<R> C;
    R P[9];
    const double psi = snh_point<R>(Fd, mud, lamd, L.level, C, P);
    r[0] = wd;
    r[1] = psi;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        r[2 + k] = Ji[k];
        r[11 + k] = L.level >= 1 ? (double)C.F[k] : 0.0;
        r[20 + k] = L.level >= 1 ? (double)C.C[k] : 0.0;
        r[29 + k] = L.level >= 1 ? (double)P[k] : 0.0;
    }
    r[38] = L.level >= 1 ? (double)C.cI : 0.0;
    r[39] = L.level >= 1 ? (double)C.cF : 0.0;
    r[40] = L.level >= 1 ? (double)C.cC : 0.0;
    r[41] = L.level >= 1 ? (double)C.cS : 0.0;
    if (proj) {
        double mlam[9], M[9][9];
        const int nm = snh_neg_modes_call(Fd, mud, lamd, mlam, M);
        double* md = B.ho_modes + ((int64_t)e * nq + q) * 91;
        md[0] = nm;
        for (int m = 0; m < nm; ++m) {
            md[1 + m] = mlam[m];
#pragma unroll
            for (int k = 0; k < 9; ++k) md[10 + 9 * m + k] = M[m][k];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128)
k_tetho_points(ElemLaunch L, int scene, int blk)
{
    const SceneDev& S = L.scenes[scene];
    if (!(S.sc == nullptr || S.sc->active)) return;
    const ElemBlock& B = S.blk[blk];
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nq = B.ho_nq;
    if (idx >= B.ho_n * nq) return;
    // consecutive threads: consecutive points of one element (the
    // element's records are contiguous)
    const int64_t e = idx / nq;
    tetho_point<R>(L, S, B, e, (int)(idx - e * nq));
}

// shared bytes of one element in k_tetho_blocks: with projection its
// modes (double), then its records and (G, F G, cof(F) G) per (point,
// node) in the element precision (rs = sizeof(R)); 16-byte multiples
__host__ __device__ constexpr int tetho_smem_bytes(int K, int nq, bool proj, int rs)
{
    return ((proj ? nq * 91 * 8 : 0) + (nq * kHoRec + nq * K * 9) * rs + 15) / 16 * 16;
}
constexpr int kHoBlockThreads = 256;

template <typename R, typename HT>
__global__ void __launch_bounds__(kHoBlockThreads)
k_tetho_blocks(ElemLaunch L, int scene, int blk, int epc)
{
    extern __shared__ __align__(16) unsigned char hsm_raw[];
    const SceneDev& S = L.scenes[scene];
    if (!(S.sc == nullptr || S.sc->active)) return;
    const ElemBlock& B = S.blk[blk];
    const int K = B.ho_K, NS = B.ho_S, nq = B.ho_nq;
    const int64_t ne = B.ho_n;
    const bool proj = L.level >= 2 && L.project;
    const int per = tetho_smem_bytes(K, nq, proj, (int)sizeof(R));
    const int tpe = kHoBlockThreads / epc;   // threads per element
    const int g = threadIdx.x / tpe, t = threadIdx.x - g * tpe;
    const int64_t e = (int64_t)blockIdx.x * epc + g;
    const bool live = g < epc && e < ne;
    double* mds = (double*)(hsm_raw + (size_t)g * per);   // [q][91] (with projection)
    R* rec = (R*)(mds + (proj ? nq * 91 : 0));             // [q][kHoRec]
    R* gv = rec + nq * kHoRec;   // [q][node][9]: G (3), F G (3), C G (3)
    // ---- the element's records (in R) and modes
    if (live) {
        const double* src = B.ho_rec + e * nq * kHoRec;
        for (int i = t; i < nq * kHoRec; i += tpe) rec[i] = (R)__ldg(src + i);
        if (proj) {
            const double* ms = B.ho_modes + e * nq * 91;
            for (int i = t; i < nq * 91; i += tpe) mds[i] = __ldg(ms + i);
        }
    }
    __syncthreads();
    // ---- G_qa, F G_qa, cof(F) G_qa (in the element precision R; G from
    // the double records)
    if (live && L.level >= 1) {
        for (int i = t; i < nq * K; i += tpe) {
            const int q = i / K, a = i - q * K;
            const double* rd = B.ho_rec + (e * nq + q) * kHoRec;
            const R* r = rec + q * kHoRec;
            const double* dn = B.ho_dN + (q * K + a) * 3;
            R Gr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Gr[c] = (R)(dn[0] * __ldg(rd + 2 + c) + dn[1] * __ldg(rd + 5 + c) +
                            dn[2] * __ldg(rd + 8 + c));
            R u[3], v[3];
            matvec3(r + 11, Gr, u);
            matvec3(r + 20, Gr, v);
            R* o = gv + (q * K + a) * 9;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o[c] = Gr[c];
                o[3 + c] = u[c];
                o[6 + c] = v[c];
            }
        }
    }
    __syncthreads();
    if (!live) return;
    int bad = 0;
    const int P = K * (K + 1) / 2;
    const int64_t sid0 = e * NS;
    // ---- owned blocks (one per thread), node gradients, energy
    for (int it = t; it < P + K + 1; it += tpe) {
        if (it < P && L.level >= 2) {
            const int* pr = B.ho_pair + 3 * it;   // nodes (in the owner's local order), slot
            const int na = pr[0], nb = pr[1], slot = pr[2];
            const bool diag = na == nb;
            R acc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = R(0);
            for (int q = 0; q < nq; ++q) {
                const R* r = rec + q * kHoRec;
                const R* ga = gv + (q * K + na) * 9;
                const R* gb = gv + (q * K + nb) * 9;
                SnhCore<R> C;
#pragma unroll
                for (int k = 0; k < 9; ++k) C.F[k] = r[11 + k];
                const R w = r[0];
                C.cI = w * r[38];
                C.cF = w * r[39];
                C.cC = w * r[40];
                C.cS = w * r[41];
                R blkv[9];
                snh_block(C, ga, gb, ga + 3, gb + 3, ga + 6, gb + 6, diag, blkv);
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] += blkv[k];
                if (proj) {
                    const double* md = mds + q * 91;
                    const int nm = (int)md[0];
                    for (int m = 0; m < nm; ++m) {
                        const double* M = md + 10 + 9 * m;
                        double wa[3], wb[3];
#pragma unroll
                        for (int rr = 0; rr < 3; ++rr) {
                            wa[rr] = M[3 * rr] * (double)ga[0] + M[3 * rr + 1] * (double)ga[1] +
                                     M[3 * rr + 2] * (double)ga[2];
                            wb[rr] = M[3 * rr] * (double)gb[0] + M[3 * rr + 1] * (double)gb[1] +
                                     M[3 * rr + 2] * (double)gb[2];
                        }
                        const double sc = __ldg(B.ho_rec + (e * nq + q) * kHoRec) * md[1 + m];
#pragma unroll
                        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                            for (int c = 0; c < 3; ++c) acc[3 * rr + c] -= (R)(sc * wa[rr] * wb[c]);
                    }
                }
            }
            const int j = slot / 10, ab = slot - 10 * (slot / 10);
#pragma unroll
            for (int k = 0; k < 9; ++k) bad |= nonfinite_bits(acc[k]) ? 1 : 0;
            if (L.out_H) {
                // the sub-stencil's full 12x12: block (a, b) and its transpose
                int la = 0, lb = 0;
                for (int x = 0; x < 4; ++x)
                    for (int y = x; y < 4; ++y)
                        if (up_index(x, y) == ab) {
                            la = x;
                            lb = y;
                        }
                double* full = L.out_H + 144 * (sid0 + j);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        full[(3 * la + i) * 12 + 3 * lb + k] = (double)acc[3 * i + k];
                        full[(3 * lb + k) * 12 + 3 * la + i] = (double)acc[3 * i + k];
                    }
            } else {
                HT* dst = (HT*)S.He + 90 * (B.base + sid0 + j) + 9 * ab;
#pragma unroll
                for (int k = 0; k < 9; ++k) dst[k] = (HT)acc[k];
            }
        } else if (it >= P && it < P + K && L.level >= 1) {
            const int a = it - P;
            const int gs = B.ho_gown[a];   // owner sub-stencil * 4 + local node
            R gl[3] = {R(0), R(0), R(0)};
            for (int q = 0; q < nq; ++q) {
                const R* r = rec + q * kHoRec;
                const R* Gr = gv + (q * K + a) * 9;
                const R w = r[0];
                const R* Pq = r + 29;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    gl[i] += w * (Pq[i * 3 + 0] * Gr[0] + Pq[i * 3 + 1] * Gr[1] + Pq[i * 3 + 2] * Gr[2]);
            }
            double* gout = L.out_g ? L.out_g + 12 * (sid0 + gs / 4)
                                   : S.ge + 12 * (B.base + sid0 + gs / 4);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                gout[3 * (gs % 4) + i] = (double)gl[i];
                bad |= nonfinite_bits(gl[i]) ? 1 : 0;
            }
        } else if (it == P + K) {
            // the energy in double from the double records
            const double* rd = B.ho_rec + e * nq * kHoRec;
            double E = 0.0;
            for (int q = 0; q < nq; ++q) E += __ldg(rd + q * kHoRec) * __ldg(rd + q * kHoRec + 1);
            bad |= nonfinite_bits(E) ? 1 : 0;
            if (L.out_E) L.out_E[sid0] = E;
            else S.Ee[B.base + sid0] = E;
        }
    }
    // ---- zeros in every slot no block owns (and the energies of j > 0)
    for (int i = t; i < NS * 10; i += tpe) {
        const int j = i / 10, ab = i - 10 * j;
        if ((B.ho_own[j] >> ab) & 1) continue;
        if (L.level < 2) break;
        if (L.out_H) {
            int la = 0, lb = 0;
            for (int x = 0; x < 4; ++x)
                for (int y = x; y < 4; ++y)
                    if (up_index(x, y) == ab) {
                        la = x;
                        lb = y;
                    }
            double* full = L.out_H + 144 * (sid0 + j);
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    full[(3 * la + ii) * 12 + 3 * lb + k] = 0.0;
                    full[(3 * lb + k) * 12 + 3 * la + ii] = 0.0;
                }
        } else {
            HT* dst = (HT*)S.He + 90 * (B.base + sid0 + j) + 9 * ab;
#pragma unroll
            for (int k = 0; k < 9; ++k) dst[k] = HT(0);
        }
    }
    for (int i = t; i < NS * 4; i += tpe) {
        const int j = i / 4, a = i - 4 * j;
        if (L.level >= 1 && !((B.ho_own[j] >> (10 + a)) & 1)) {
            double* gout = L.out_g ? L.out_g + 12 * (sid0 + j) : S.ge + 12 * (B.base + sid0 + j);
#pragma unroll
            for (int k = 0; k < 3; ++k) gout[3 * a + k] = 0.0;
        }
        if (a == 0 && j > 0) {
            if (L.out_E) L.out_E[sid0 + j] = 0.0;
            else S.Ee[B.base + sid0 + j] = 0.0;
        }
    }
    if (bad) B.ho_flag[e] = 1;
}

// The element kernel's share of a high-order tile (kHoTileElems whole
// elements): the energies and non-finite flags the two launches before it
// left, summed in element order.
template <typename R, typename HT>
__device__ void tetho_tile(const ElemLaunch& L, const SceneDev& S, const ElemBlock& B,
                           const Tile& T, ThreadOut& o)
{
    const int NS = B.ho_S;
    const int64_t e0 = T.start / NS;
    const int nel = T.count / NS;
    o.E = 0.0;
    if ((int)threadIdx.x < nel) {
        const int64_t e = e0 + threadIdx.x;
        o.E = L.out_E ? L.out_E[e * NS] : S.Ee[B.base + e * NS];
        if (B.ho_flag[e]) {
            o.nonfinite = 1;
            B.ho_flag[e] = 0;
        }
    }
}

template <typename R, typename HT>
__device__ void eval_hinge(const ElemLaunch& L, const SceneDev& S, const ElemBlock& B,
                           int64_t e, ThreadOut& o)
{
    const int4 t = B.conn[e];
    const int nid[4] = {t.x, t.y, t.z, t.w};
    // s = sum_a q_a x_a, formed relative to node 0 (exact for any q once the
    // q-sum term is added back; for a translation-free hinge it vanishes)
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
    const double kcd = B.kb * B.c[e];
    o.E = 0.5 * kcd * (sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
    if (nonfinite_bits(o.E)) o.nonfinite = 1;
    const R kc = (R)kcd;
    const R s[3] = {(R)sd[0], (R)sd[1], (R)sd[2]};
    R q[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] = (R)qd[a];
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
        write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
    }
}

template <typename R, typename HT>
__device__ void eval_barrier(const ElemLaunch& L, int scene, int blk, const SceneDev& S,
                             const ElemBlock& B, int64_t e, ThreadOut& o)
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
        // the energy (the line-search quantity) is always evaluated in double
        BarrierOut<double> bd;
        const int sd = barrier_eval<double>(xr, B.dhat, B.kappa, 0, bd);
        Ed = (sd == 1) ? bd.E : 0.0;
        if (sd != 1) st = sd;
    }
    const int64_t gid = B.base + e;
    if (st < 0) o.bad = 1;
    o.E = (st == 1) ? Ed : 0.0;
    if (nonfinite_bits(o.E)) o.nonfinite = 1;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) gout[k] = (st == 1) ? to_f64_bits(bo.g[k]) : 0.0;
    }
    if (L.level >= 2) {
        auto blockfn = [&](int a, int b, R* out) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    out[i * 3 + k] = (st == 1) ? bo.H[(3 * a + i) * 12 + 3 * b + k] : R(0);
        };
        HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
        double* full = L.out_H ? L.out_H + 144 * e : nullptr;
        write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
        if (st == 1 && L.project) {
            // M = (Hd kron I3) H (Hd kron I3) restricted to the modes c, d = 1..3
            double M[45];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    double Tm[4][3];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        double h[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            h[b] = 0.5 * (to_f64_bits(bo.H[(3 * a + i) * 12 + 3 * b + k]) +
                                          to_f64_bits(bo.H[(3 * b + k) * 12 + 3 * a + i]));
                        had_fwd(h[0], h[1], h[2], h[3], Tm[a][0], Tm[a][1], Tm[a][2]);
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        double y[3];
                        had_fwd(Tm[0][d], Tm[1][d], Tm[2][d], Tm[3][d], y[0], y[1], y[2]);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            if (3 * c + i >= 3 * d + k) M[pk(3 * c + i, 3 * d + k)] = y[c];
                    }
                }
            o.clamped = queue_if_indefinite(L, scene, blk, e, M);
        }
    }
}

// KINDS: bit mask of the stencil kinds compiled in (1 SNH, 2 hinge, 4
// barrier), 8 for the F-space projection of the SNH tets (project mode
// 2), 16 for tets of the other densities, 32 for friction and 64 for
// high-order tets. A batch with SNH tets only
// runs an SNH-only instantiation, which needs fewer registers than the one
// that can take every kind.
template <typename R, typename HT, int KINDS>
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
            bool ho = false;
            if constexpr ((KINDS & 64) != 0) {
                if (B.kind == SX_KIND_TET_HO) {
                    // block-uniform: every thread takes part (the tile synchronizes)
                    ho = true;
                    tetho_tile<R, HT>(L, S, B, T, o);   // writes its sub-stencils' energies
                }
            }
            if (!ho && (int)threadIdx.x < T.count) {
                const int64_t e = T.start + threadIdx.x;
                if ((KINDS & 16) && B.kind == SX_KIND_SNH_TET4 && B.model != SX_MODEL_SNH)
                    eval_model<R, HT>(L, T.scene, T.blk, S, B, e, o);
                else if ((KINDS & 1) && B.kind == SX_KIND_SNH_TET4)
                    eval_snh<R, HT, (KINDS & 8) != 0>(L, T.scene, T.blk, S, B, e, o);
                else if ((KINDS & 2) && B.kind == SX_KIND_HINGE4)
                    eval_hinge<R, HT>(L, S, B, e, o);
                else if ((KINDS & 32) && B.kind == SX_KIND_PT_FRICTION)
                    eval_friction<R, HT>(L, S, B, e, o);
                else if ((KINDS & 4) && B.kind == SX_KIND_PT_BARRIER)
                    eval_barrier<R, HT>(L, T.scene, T.blk, S, B, e, o);
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

// host-side access to the instantiations of one translation unit
template <int K>
const void* elements_kernel_ptr(bool f32)
{
    return f32 ? (const void*)k_elements<float, float, K> : (const void*)k_elements<double, double, K>;
}

template <int K>
void elements_launch(bool f32, const ElemLaunch& L, int grid, cudaStream_t s)
{
    if (f32) k_elements<float, float, K><<<grid, kElemThreads, 0, s>>>(L);
    else k_elements<double, double, K><<<grid, kElemThreads, 0, s>>>(L);
}

}  // namespace sx
