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

#include <algorithm>
#include <atomic>

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

int elements_block_threads() { return kElemThreads; }
int clamp_block_threads() { return kClampThreads; }

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
        // P = a F + b cof F. Its two O(mu') parts cancel at rest, so it is
        // formed from D = F - I: cof(I + D) = I + (tr D) I - D^T + cof D gives
        // P = (a + b) I + a D + b ((tr D) I - D^T + cof D), where
        // a + b = mu' Ic3 / (4 (Ic + 1)) + lam' (J - 1) (alpha = 1 + 3 mu' / (4 lam'))
        // is taken in double; the rest is O(mu' |D|) and keeps R's relative
        // precision (in FP32 this is what lets the assembled forces resolve
        // below float epsilon times mu')
        const double Icd = 3.0 + Ic3;
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

// 9x9 translation-free Hessian M (double, packed lower) of an SNH tet.
template <typename R>
__device__ __forceinline__ void snh_M(const SnhCore<R>& S, double (&M)[45])
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
                for (int k = 0; k < 3; ++k)
                    if (3 * d + k <= 3 * c + i || c != d)
                        M[pk(3 * d + k, 3 * c + i)] = (double)blk[i * 3 + k];
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
            for (int k = 0; k < 9; ++k) bad |= !isfinite((double)blk[k]);
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

// project mode 2 for one SNH tet: removes from its Hessian blocks the
// negative modes of d2psi/dF2 (H = V B^T proj(d2psi/dF2) B). In the frame
// of the signed SVD F = U diag(s) V^T (U, V rotations) the material Hessian
// a I + gam F F^T + lam' C C^T + b dC/dF splits into three twist/flip pairs,
// eigenvalue a - b s_k on (u_i v_j^T + u_j v_i^T)/sqrt2 and a + b s_k on
// (u_i v_j^T - u_j v_i^T)/sqrt2 ({i, j, k} = {0, 1, 2}), and the stretch
// block a I + gam s s^T + lam' p p^T + b K on U diag(q) V^T, with
// p = (s1 s2, s0 s2, s0 s1) and K the symmetric 3x3 with zero diagonal and
// K01 = s2, K02 = s1, K12 = s0. A negative mode (lambda, E) changes block
// (a, b) by -V lambda (E G_a)(E G_b)^T. Returns the number of modes removed.
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
    // g[a][k] = v_k . G_a
    double G[4][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        G[1][j] = Dinv[j];
        G[2][j] = Dinv[3 + j];
        G[3][j] = Dinv[6 + j];
        G[0][j] = -(Dinv[j] + Dinv[3 + j] + Dinv[6 + j]);
    }
    double g[4][3];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            g[n][k] = G[n][0] * Vm[k] + G[n][1] * Vm[3 + k] + G[n][2] * Vm[6 + k];
    int removed = 0;
    auto remove = [&](double lambda, const double (&w)[12]) {
        const double sc = Vd * lambda;
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
        ++removed;
    };
    const double h = 0.70710678118654752440;   // 1/sqrt(2)
    // twist / flip pairs
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
#pragma unroll
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            const double lambda = a + sgn * b * sg[k];   // sgn -1: symmetric, +1: antisymmetric
            if (!(lambda < 0.0)) continue;
            const double sym = (sgn < 0) ? 1.0 : -1.0;
            double w[12];
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    w[3 * n + r] = h * (U[i][r] * g[n][j] + sym * U[j][r] * g[n][i]);
            remove(lambda, w);
        }
    }
    // stretch block
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
        double w[12];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int r = 0; r < 3; ++r)
                w[3 * n + r] = Q3[0 + e] * g[n][0] * U[0][r] + Q3[3 + e] * g[n][1] * U[1][r] +
                               Q3[6 + e] * g[n][2] * U[2][r];
        remove(lambda, w);
    }
    return removed;
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
        {
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
            write_blocks<R, HT>(blockfn, staged, full, &o.nonfinite);
        }
        if (FPROJ && L.project == 2) {
            HT* staged = L.out_H ? nullptr : (HT*)S.He + 90 * gid;
            double* full = L.out_H ? L.out_H + 144 * e : nullptr;
            o.clamped = snh_fproj<HT>(xg, Dinv, B.V[e], B.mu[e], B.lam[e], staged, full) > 0;
        } else if (L.project) {
            double M[45];
            snh_M<R>(C, M);
            o.clamped = queue_if_indefinite(L, scene, blk, e, M);
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
    if (!isfinite(o.E)) o.nonfinite = 1;
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
    if (!isfinite(o.E)) o.nonfinite = 1;
    if (L.level >= 1) {
        double* gout = L.out_g ? L.out_g + 12 * e : S.ge + 12 * gid;
#pragma unroll
        for (int k = 0; k < 12; ++k) gout[k] = (st == 1) ? (double)bo.g[k] : 0.0;
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
                            h[b] = 0.5 * ((double)bo.H[(3 * a + i) * 12 + 3 * b + k] +
                                          (double)bo.H[(3 * b + k) * 12 + 3 * a + i]);
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
// barrier), and 8 for the F-space projection of the SNH tets (project mode
// 2). A batch with SNH tets only runs an SNH-only instantiation, which needs
// fewer registers than the one that can take every kind.
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
            if ((int)threadIdx.x < T.count) {
                const int64_t e = T.start + threadIdx.x;
                if ((KINDS & 1) && B.kind == SX_KIND_SNH_TET4)
                    eval_snh<R, HT, (KINDS & 8) != 0>(L, T.scene, T.blk, S, B, e, o);
                else if ((KINDS & 2) && B.kind == SX_KIND_HINGE4)
                    eval_hinge<R, HT>(L, S, B, e, o);
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

// The projection of a batched evaluation in two launches. The float part
// runs per queued stencil and bins the stencil by k (the size of its N
// block, 0..9); the double part then takes the stencils bucket by bucket,
// so the 32 stencils of a warp share k and the warp runs only the rotations
// they all need. Every stencil's arithmetic is the same as in k_clamp.
template <int NT>
__global__ void __launch_bounds__(NT)
k_clamp_float(ElemLaunch L)
{
    const int count = min(*L.clamp_count, L.clamp_cap);
    const int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (idx >= count) return;
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
    float* Xg = L.clamp_X;   // [81][cap], entry r*9 + slot of stencil idx
    const int k = eig9_float(Mg, fro, [&](int r, int slot, float v) {
        Xg[(int64_t)(r * 9 + slot) * cap + idx] = v;
    });
    L.clamp_fro[idx] = fro;
    // bucket slot: one atomic per (warp, k) for the lanes that share k
    const unsigned peers = __match_any_sync(__activemask(), k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(L.clamp_bucket_count + k, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int pos = base + __popc(peers & ((1u << lane) - 1u));
    L.clamp_bucket[(int64_t)k * cap + pos] = (int)idx;
}

template <typename HT, int NT>
__global__ void __launch_bounds__(NT)
k_clamp_double(ElemLaunch L)
{
    extern __shared__ __align__(16) double Xs[];   // [81][NT]
    const SmemMat X{Xs + threadIdx.x, NT};
    __shared__ int s_k, s_off;
    if (threadIdx.x == 0) {
        // block -> (bucket, offset): buckets in order, ceil(count / NT) blocks each
        int b = blockIdx.x;
        s_k = -1;
        s_off = 0;
        for (int kk = 0; kk < 10; ++kk) {
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
    if (k < 0) return;
    const int cntk = L.clamp_bucket_count[k];
    const int jj = s_off + threadIdx.x;
    const unsigned live = __ballot_sync(0xffffffffu, jj < cntk);
    if (jj >= cntk) return;
    const int64_t cap = L.clamp_cap;
    const int64_t idx = L.clamp_bucket[(int64_t)k * cap + jj];
    const float* Xg = L.clamp_X;
#pragma unroll
    for (int q = 0; q < 81; ++q) X(q / 9, q % 9) = (double)Xg[(int64_t)q * cap + idx];
    const ClampRef ref = L.clamp_ref[idx];
    const double* Mg = L.clamp_M + 45 * idx;
    const double fro = L.clamp_fro[idx];
    const double tau = 1e-13 * fro;
    double lam[9];
    eig9_double(Mg, X, lam, fro, sizeof(HT) == 4 ? SX_CLAMP_THETA32 : 1e-13, k, live);
    clamp_finish<HT>(L, ref, Mg, X, lam, k, tau, live);
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

const void* elements_kernel(int precision, int variant)
{
    const bool f = precision == SX_FP32;
    switch (variant) {
    case 1: return f ? (const void*)k_elements<float, float, 1> : (const void*)k_elements<double, double, 1>;
    case 2: return f ? (const void*)k_elements<float, float, 15> : (const void*)k_elements<double, double, 15>;
    case 3: return f ? (const void*)k_elements<float, float, 9> : (const void*)k_elements<double, double, 9>;
    default: return f ? (const void*)k_elements<float, float, 7> : (const void*)k_elements<double, double, 7>;
    }
}

int elements_variant(int kinds, int project)
{
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
            err = cudaMemsetAsync(L.clamp_bucket_count, 0, 10 * sizeof(int), s);
        if (err != cudaSuccess) return err;
    }
    const int v = elements_variant(L.kinds, L.level >= 2 ? L.project : 0);
    if (L.precision == SX_FP32) {
        if (v == 1) k_elements<float, float, 1><<<grid, kElemThreads, 0, s>>>(L);
        else if (v == 2) k_elements<float, float, 15><<<grid, kElemThreads, 0, s>>>(L);
        else if (v == 3) k_elements<float, float, 9><<<grid, kElemThreads, 0, s>>>(L);
        else k_elements<float, float, 7><<<grid, kElemThreads, 0, s>>>(L);
    } else {
        if (v == 1) k_elements<double, double, 1><<<grid, kElemThreads, 0, s>>>(L);
        else if (v == 2) k_elements<double, double, 15><<<grid, kElemThreads, 0, s>>>(L);
        else if (v == 3) k_elements<double, double, 9><<<grid, kElemThreads, 0, s>>>(L);
        else k_elements<double, double, 7><<<grid, kElemThreads, 0, s>>>(L);
    }
    return cudaGetLastError();
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
        attr_done.fetch_or(bit, std::memory_order_release);
    }
    const bool f32 = L.precision == SX_FP32;
    if (L.clamp_X) {
        // two launches: float part binned by k, then the double part per bucket
        const int64_t cap = L.clamp_cap;
        const int ga = (int)std::max<int64_t>(1, (cap + 127) / 128);
        k_clamp_float<128><<<ga, 128, 0, s>>>(L);
        const int gb = (int)std::max<int64_t>(1, (cap + nt - 1) / nt + 10);
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
