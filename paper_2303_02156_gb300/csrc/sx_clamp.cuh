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
// of M. The 9x9 problem is solved in double precision:
//   1. shifted LDL^T of M + tau I (tau = 1e-13 ||M||_F): if it succeeds
//      the stencil is left as is (the change is at most tau);
//   2. otherwise Householder reduction to tridiagonal T = Q^T M Q,
//      eigenvalues of T by implicit QL with Wilkinson shifts, and for each
//      eigenvalue below -tau an eigenvector by inverse iteration on T
//      (partial-pivoting LU, three sweeps, Gram-Schmidt inside clusters),
//      mapped back through the reflectors.
// All steps are textbook dense symmetric eigen-methods (Golub & Van Loan,
// ch. 8); the result, a spectral function of H, is unique even where
// eigenvectors are not.
#pragma once

#include <float.h>
#include <math.h>

namespace sx {

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

// Eigenvalues of the symmetric tridiagonal (d, e), e[0..n-2] the
// subdiagonal, by implicit QL with Wilkinson shifts. d is overwritten by
// the eigenvalues (unordered). Returns false if an eigenvalue needed more
// than 60 sweeps.
__device__ inline bool ql_eigvals9(double* d, double* e, double abs_floor)
{
    const int n = 9;
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m) {
                double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= DBL_EPSILON * dd || fabs(e[m]) <= abs_floor) break;
            }
            if (m == l) break;
            if (++iter > 60) return false;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            bool restart = false;
            for (int i = m - 1; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    restart = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return true;
}

// Negative eigenpairs of the symmetric 9x9 A (row-major, both triangles;
// destroyed). Writes up to 9 pairs (lam[k] < -tau ascending, V[k][0..8]
// orthonormal) and returns their number; returns -1 if QL failed (the
// caller reports it). `fro_out` receives ||A||_F.
__device__ inline int neg_eigs9(double* A, double* lam, double* V, double* fro_out)
{
    const int n = 9;
    double fro2 = 0.0;
#pragma unroll
    for (int i = 0; i < 81; ++i) fro2 = fma(A[i], A[i], fro2);
    double fro = sqrt(fro2);
    *fro_out = fro;
    if (fro == 0.0) return 0;
    const double tau = 1e-13 * fro;

    // 1. shifted LDL^T test (no pivoting: succeeds iff A + tau I is PD)
    {
        double L[81];
        double dg[9];
        bool pd = true;
        for (int j = 0; j < n && pd; ++j) {
            double s = A[j * 9 + j] + tau;
            for (int k = 0; k < j; ++k) s -= L[j * 9 + k] * L[j * 9 + k] * dg[k];
            if (!(s > 0.0)) {
                pd = false;
                break;
            }
            dg[j] = s;
            double inv = 1.0 / s;
            for (int i = j + 1; i < n; ++i) {
                double t = A[i * 9 + j];
                for (int k = 0; k < j; ++k) t -= L[i * 9 + k] * L[j * 9 + k] * dg[k];
                L[i * 9 + j] = t * inv;
            }
        }
        if (pd) return 0;
    }

    // 2. Householder tridiagonalization on the lower triangle; reflector k
    //    (acting on rows k+1..8) is kept in column k below the diagonal.
    double d[9], e[9], beta[9];
    for (int k = 0; k < n - 2; ++k) {
        double a2 = 0.0;
        for (int i = k + 1; i < n; ++i) a2 = fma(A[i * 9 + k], A[i * 9 + k], a2);
        double xn = sqrt(a2);
        double x0 = A[(k + 1) * 9 + k];
        if (xn <= 1e-300) {
            beta[k] = 0.0;
            e[k] = x0;
            continue;
        }
        double alpha = (x0 > 0.0) ? -xn : xn;
        double v0 = x0 - alpha;
        double b = 1.0 / (xn * (xn + fabs(x0)));   // 2 / v^T v
        A[(k + 1) * 9 + k] = v0;
        beta[k] = b;
        e[k] = alpha;
        // p = b * A' v on the trailing block, lower storage
        double p[9];
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j <= i; ++j) s = fma(A[i * 9 + j], A[j * 9 + k], s);
            for (int j = i + 1; j < n; ++j) s = fma(A[j * 9 + i], A[j * 9 + k], s);
            p[i] = b * s;
            K = fma(A[i * 9 + k], p[i], K);
        }
        K *= 0.5 * b;
        for (int i = k + 1; i < n; ++i) p[i] = fma(-K, A[i * 9 + k], p[i]);   // w
        for (int i = k + 1; i < n; ++i) {
            double vi = A[i * 9 + k], wi = p[i];
            for (int j = k + 1; j <= i; ++j)
                A[i * 9 + j] -= fma(vi, p[j], wi * A[j * 9 + k]);
        }
    }
    for (int i = 0; i < n; ++i) d[i] = A[i * 9 + i];
    e[n - 2] = A[(n - 1) * 9 + (n - 2)];

    // 3. eigenvalues of T
    double ev[9], ee[9];
    for (int i = 0; i < n; ++i) { ev[i] = d[i]; ee[i] = e[i]; }
    if (!ql_eigvals9(ev, ee, 1e-18 * fro)) return -1;

    // 4. the ones below -tau, ascending
    int k = 0;
    for (int i = 0; i < n; ++i)
        if (ev[i] < -tau) {
            double v = ev[i];
            int j = k++;
            while (j > 0 && lam[j - 1] > v) { lam[j] = lam[j - 1]; --j; }
            lam[j] = v;
        }
    if (k == 0) return 0;

    // 5. inverse iteration on T for each, then back through the reflectors
    const double tiny = DBL_EPSILON * fro;
    for (int t = 0; t < k; ++t) {
        const double sig = lam[t];
        // LU with partial pivoting of T - sig I
        double a[9], bsup[9], u2[9], m[9], rinv[9];
        unsigned piv = 0u;
        for (int i = 0; i < n; ++i) {
            a[i] = d[i] - sig;
            bsup[i] = (i < n - 1) ? e[i] : 0.0;
            u2[i] = 0.0;
        }
        for (int i = 0; i < n - 1; ++i) {
            double c = e[i];   // subdiagonal of row i+1
            if (fabs(a[i]) >= fabs(c)) {
                if (fabs(a[i]) < tiny) a[i] = copysign(tiny, a[i] == 0.0 ? 1.0 : a[i]);
                m[i] = c / a[i];
                a[i + 1] -= m[i] * bsup[i];
            } else {
                piv |= 1u << i;
                double mi = a[i] / c;
                m[i] = mi;
                double na_i = c, nb_i = a[i + 1];
                double nu2 = (i + 1 < n - 1) ? bsup[i + 1] : 0.0;
                double na_i1 = bsup[i] - mi * a[i + 1];
                double nb_i1 = (i + 1 < n - 1) ? -mi * bsup[i + 1] : 0.0;
                a[i] = na_i;
                bsup[i] = nb_i;
                u2[i] = nu2;
                a[i + 1] = na_i1;
                if (i + 1 < n - 1) bsup[i + 1] = nb_i1;
            }
        }
        if (fabs(a[n - 1]) < tiny) a[n - 1] = copysign(tiny, a[n - 1] == 0.0 ? 1.0 : a[n - 1]);
        for (int i = 0; i < n; ++i) rinv[i] = 1.0 / a[i];

        double y[9];
        for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.618033988749895 * (double)((i * 7 + t * 3) % 9);
        for (int sweep = 0; sweep < 3; ++sweep) {
            // orthogonalize against earlier vectors of the same cluster
            for (int s = 0; s < t; ++s) {
                if (fabs(lam[s] - sig) > 1e-3 * fro) continue;
                double dt_ = 0.0;
                for (int i = 0; i < n; ++i) dt_ = fma(V[s * 9 + i], y[i], dt_);
                for (int i = 0; i < n; ++i) y[i] = fma(-dt_, V[s * 9 + i], y[i]);
            }
            // forward elimination on the rhs
            for (int i = 0; i < n - 1; ++i) {
                if (piv & (1u << i)) { double tmp = y[i]; y[i] = y[i + 1]; y[i + 1] = tmp; }
                y[i + 1] -= m[i] * y[i];
            }
            // back substitution
            y[n - 1] *= rinv[n - 1];
            y[n - 2] = (y[n - 2] - bsup[n - 2] * y[n - 1]) * rinv[n - 2];
            for (int i = n - 3; i >= 0; --i)
                y[i] = (y[i] - bsup[i] * y[i + 1] - u2[i] * y[i + 2]) * rinv[i];
            double nn = 0.0;
            for (int i = 0; i < n; ++i) nn = fma(y[i], y[i], nn);
            double inv = 1.0 / sqrt(nn);
            for (int i = 0; i < n; ++i) y[i] *= inv;
        }
        // final orthogonalization inside the cluster
        for (int s = 0; s < t; ++s) {
            if (fabs(lam[s] - sig) > 1e-3 * fro) continue;
            double dt_ = 0.0;
            for (int i = 0; i < n; ++i) dt_ = fma(V[s * 9 + i], y[i], dt_);
            for (int i = 0; i < n; ++i) y[i] = fma(-dt_, V[s * 9 + i], y[i]);
            double nn = 0.0;
            for (int i = 0; i < n; ++i) nn = fma(y[i], y[i], nn);
            double inv = 1.0 / sqrt(nn);
            for (int i = 0; i < n; ++i) y[i] *= inv;
        }
        for (int i = 0; i < n; ++i) V[t * 9 + i] = y[i];
    }
    // back-transform all vectors: v = H_0 H_1 ... H_6 w
    for (int t = 0; t < k; ++t) {
        double* w = V + t * 9;
        for (int kk = n - 3; kk >= 0; --kk) {
            if (beta[kk] == 0.0) continue;
            double s = 0.0;
            for (int i = kk + 1; i < n; ++i) s = fma(A[i * 9 + kk], w[i], s);
            s *= beta[kk];
            for (int i = kk + 1; i < n; ++i) w[i] = fma(-s, A[i * 9 + kk], w[i]);
        }
    }
    return k;
}

}  // namespace sx
