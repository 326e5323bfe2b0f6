// sx_barrier.cuh -- point-triangle IPC barrier (§6.4, Eq. 15) on the
// unsigned point-triangle distance d, active only for 0 < d < dhat
// (conditional evaluation, §5.2 Eq. 9).
//
// Route: coordinates arrive relative to the point p (formed in double),
// are scaled by the largest point-vertex distance ell so that every
// intermediate is O(1) in float, and the closest feature is found from the
// barycentric coordinates of the plane projection (face) or, outside the
// triangle, from the nearest of the three clamped segment projections
// (edge interior or end vertex). Per feature, with z the feature's edge
// vectors:
//   face   z = (e, E1, E2), e = p - a, E1 = b - a, E2 = c - a,
//          N = E1 x E2, u = e.N, w = N.N, d = |u| / sqrt(w);
//   edge   z = (e, E), e = p - u, E = w - u,
//          s = e.e - (e.E)^2/(E.E), d = sqrt(s);
//   vertex z = r = p - v, d = |r|;
// gradient and Hessian in z are closed forms, mapped to the 12 stencil
// coordinates by the fixed +-1 incidence of z on (p, t0, t1, t2). Then
// E = b(d), g = b'(d) grad d, H = b''(d) grad d grad d^T + b'(d) hess d with
// b(d) = -kappa (d - dhat)^2 ln(d / dhat).
#pragma once

#include <math.h>

namespace sx {

template <typename R>
struct BarrierOut {
    R E;
    R g[12];
    R H[144];
};

template <typename R>
__device__ __forceinline__ R dot3(const R* a, const R* b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename R>
__device__ __forceinline__ void xprod(const R* u, const R* v, R* w)
{
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

__host__ __device__ constexpr int lc(int i, int j, int k)
{
    return (i - j) * (j - k) * (k - i) / 2;
}

// Returns 1 active, 0 inactive (d >= dhat), -1 invalid (d <= 0). xr holds
// (p, t0, t1, t2) relative to p (so xr[0..2] = 0).
template <typename R>
__device__ int barrier_eval(const double* xr, R dhat, R kappa, int level, BarrierOut<R>& o)
{
    double l2 = 0.0;
    for (int k = 1; k < 4; ++k) {
        double q = xr[3 * k] * xr[3 * k] + xr[3 * k + 1] * xr[3 * k + 1] +
                   xr[3 * k + 2] * xr[3 * k + 2];
        l2 = q > l2 ? q : l2;
    }
    if (!(l2 > 0.0)) return -1;
    const double elld = sqrt(l2);
    const R ell = (R)elld;
    R t[3][3];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) t[k][i] = (R)(xr[3 * (k + 1) + i] / elld);

    // --- closest feature -------------------------------------------------
    R E1[3], E2[3], e[3], N[3];
    for (int i = 0; i < 3; ++i) {
        E1[i] = t[1][i] - t[0][i];
        E2[i] = t[2][i] - t[0][i];
        e[i] = -t[0][i];
    }
    xprod(E1, E2, N);
    const R w = dot3(N, N);
    int feat = -1;   // 0..2 vertex, 3 = edge t0t1, 4 = t1t2, 5 = t2t0, 6 = face
    if (w > R(0)) {
        R c1[3], c2[3];
        xprod(e, E2, c1);
        xprod(E1, e, c2);
        R b1 = dot3(c1, N) / w, b2 = dot3(c2, N) / w;
        R b0 = R(1) - b1 - b2;
        if (b0 >= R(0) && b1 >= R(0) && b2 >= R(0)) feat = 6;
    }
    int eu = 0, ew = 1;
    if (feat < 0) {
        R best = R(0);
        R bestt = R(0);
        int bi = -1;
        for (int s = 0; s < 3; ++s) {
            const int iu = s, iw = (s + 1) % 3;
            R ee[3], EE[3];
            for (int i = 0; i < 3; ++i) {
                ee[i] = -t[iu][i];
                EE[i] = t[iw][i] - t[iu][i];
            }
            R bb = dot3(EE, EE);
            R tt = bb > R(0) ? dot3(ee, EE) / bb : R(0);
            tt = tt < R(0) ? R(0) : (tt > R(1) ? R(1) : tt);
            R r[3];
            for (int i = 0; i < 3; ++i) r[i] = ee[i] - tt * EE[i];
            R dd = dot3(r, r);
            if (bi < 0 || dd < best) {
                best = dd;
                bestt = tt;
                bi = s;
            }
        }
        eu = bi;
        ew = (bi + 1) % 3;
        if (bestt <= R(0)) feat = eu;
        else if (bestt >= R(1)) feat = ew;
        else feat = 3 + bi;
    }

    // --- d, grad d, hess d in z-space ------------------------------------
    int nb;          // z blocks
    int coef[4][3];  // incidence of z blocks on (p, t0, t1, t2)
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) coef[a][i] = 0;
    R d;
    R gz[9];
    R Hz[81];
    if (feat == 6) {
        nb = 3;
        coef[0][0] = 1;
        coef[1][0] = -1; coef[1][1] = -1; coef[1][2] = -1;
        coef[2][1] = 1;
        coef[3][2] = 1;
        const R u = dot3(e, N);
        if (!(u != R(0))) return -1;
        const R sg = u > R(0) ? R(1) : R(-1);
        const R rs = R(1) / sqrt(w);
        const R wi = R(1) / w;
        d = sg * u * rs;
        if (level >= 1) {
            // A1[i][j] = dN_i/dE1_j, A2[i][k] = dN_i/dE2_k
            R A1[3][3], A2[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    R s1 = R(0), s2 = R(0);
                    for (int m = 0; m < 3; ++m) {
                        if (lc(i, j, m)) s1 += R(lc(i, j, m)) * E2[m];
                        if (lc(i, m, j)) s2 += R(lc(i, m, j)) * E1[m];
                    }
                    A1[i][j] = s1;
                    A2[i][j] = s2;
                }
            R gu[9], gw[9];
            for (int j = 0; j < 3; ++j) {
                gu[j] = N[j];
                gu[3 + j] = A1[0][j] * e[0] + A1[1][j] * e[1] + A1[2][j] * e[2];
                gu[6 + j] = A2[0][j] * e[0] + A2[1][j] * e[1] + A2[2][j] * e[2];
                gw[j] = R(0);
                gw[3 + j] = R(2) * (A1[0][j] * N[0] + A1[1][j] * N[1] + A1[2][j] * N[2]);
                gw[6 + j] = R(2) * (A2[0][j] * N[0] + A2[1][j] * N[1] + A2[2][j] * N[2]);
            }
            const R c_w = R(0.5) * u * rs * wi;
            for (int k = 0; k < 9; ++k) gz[k] = sg * (rs * gu[k] - c_w * gw[k]);
            if (level >= 2) {
                R Hu[81], Hw[81];
                for (int k = 0; k < 81; ++k) { Hu[k] = R(0); Hw[k] = R(0); }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        // d2u/de dE1 = A1, d2u/de dE2 = A2, d2u/dE1_j dE2_k = e_i eps_ijk
                        Hu[(0 + i) * 9 + 3 + j] = A1[i][j];
                        Hu[(3 + j) * 9 + 0 + i] = A1[i][j];
                        Hu[(0 + i) * 9 + 6 + j] = A2[i][j];
                        Hu[(6 + j) * 9 + 0 + i] = A2[i][j];
                        R s = R(0), sn = R(0);
                        for (int m = 0; m < 3; ++m)
                            if (lc(m, i, j)) {
                                s += R(lc(m, i, j)) * e[m];
                                sn += R(lc(m, i, j)) * N[m];
                            }
                        Hu[(3 + i) * 9 + 6 + j] = s;
                        Hu[(6 + j) * 9 + 3 + i] = s;
                        // d2w = 2 (dN)^T dN + 2 N_m d2N_m
                        R h11 = R(0), h22 = R(0), h12 = R(0);
                        for (int m = 0; m < 3; ++m) {
                            h11 += A1[m][i] * A1[m][j];
                            h22 += A2[m][i] * A2[m][j];
                            h12 += A1[m][i] * A2[m][j];
                        }
                        Hw[(3 + i) * 9 + 3 + j] = R(2) * h11;
                        Hw[(6 + i) * 9 + 6 + j] = R(2) * h22;
                        Hw[(3 + i) * 9 + 6 + j] = R(2) * (h12 + sn);
                        Hw[(6 + j) * 9 + 3 + i] = R(2) * (h12 + sn);
                    }
                const R k1 = R(0.5) * rs * wi, k2 = R(0.75) * u * rs * wi * wi;
                for (int a = 0; a < 9; ++a)
                    for (int b = 0; b < 9; ++b)
                        Hz[a * 9 + b] =
                            sg * (rs * Hu[a * 9 + b] - k1 * (gu[a] * gw[b] + gw[a] * gu[b]) -
                                  c_w * Hw[a * 9 + b] + k2 * gw[a] * gw[b]);
            }
        }
    } else if (feat >= 3) {
        nb = 2;
        const int iu = eu, iw = ew;
        coef[0][0] = 1;
        coef[1 + iu][0] = -1; coef[1 + iu][1] = -1;
        coef[1 + iw][1] = 1;
        R ee[3], EE[3];
        for (int i = 0; i < 3; ++i) {
            ee[i] = -t[iu][i];
            EE[i] = t[iw][i] - t[iu][i];
        }
        const R beta = dot3(EE, EE);
        const R tt = dot3(ee, EE) / beta;
        R r[3];
        for (int i = 0; i < 3; ++i) r[i] = ee[i] - tt * EE[i];
        const R s = dot3(r, r);
        if (!(s > R(0))) return -1;
        d = sqrt(s);
        if (level >= 1) {
            const R id = R(1) / d;
            for (int i = 0; i < 3; ++i) {
                gz[i] = r[i] * id;             // ds/de / (2d) = r/d
                gz[3 + i] = -tt * r[i] * id;   // ds/dE / (2d) = -t r/d
            }
            if (level >= 2) {
                const R ib = R(1) / beta;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        const R dij = (i == j) ? R(1) : R(0);
                        R hee = R(2) * dij - R(2) * EE[i] * EE[j] * ib;
                        R heE = -R(2) * EE[i] * ee[j] * ib - R(2) * tt * dij +
                                R(4) * tt * EE[i] * EE[j] * ib;
                        R hEE = -R(2) * ee[i] * ee[j] * ib + R(4) * tt * ee[i] * EE[j] * ib +
                                R(4) * tt * EE[i] * ee[j] * ib + R(2) * tt * tt * dij -
                                R(8) * tt * tt * EE[i] * EE[j] * ib;
                        Hz[i * 9 + j] = hee;
                        Hz[i * 9 + 3 + j] = heE;
                        Hz[(3 + j) * 9 + i] = heE;
                        Hz[(3 + i) * 9 + 3 + j] = hEE;
                    }
                // hess d = hess s / (2d) - grad d grad d^T / d
                for (int a = 0; a < 6; ++a)
                    for (int b = 0; b < 6; ++b)
                        Hz[a * 9 + b] = R(0.5) * id * Hz[a * 9 + b] - id * gz[a] * gz[b];
            }
        }
    } else {
        nb = 1;
        const int iv = feat;
        coef[0][0] = 1;
        coef[1 + iv][0] = -1;
        R r[3] = {-t[iv][0], -t[iv][1], -t[iv][2]};
        const R s = dot3(r, r);
        if (!(s > R(0))) return -1;
        d = sqrt(s);
        if (level >= 1) {
            const R id = R(1) / d;
            for (int i = 0; i < 3; ++i) gz[i] = r[i] * id;
            if (level >= 2)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        Hz[i * 9 + j] = ((i == j) ? id : R(0)) - gz[i] * gz[j] * id;
        }
    }

    // --- barrier ----------------------------------------------------------
    const R dd = d * ell;   // true distance
    if (!(dd > R(0))) return -1;
    if (!(dd < dhat)) return 0;
    const R rr = dd - dhat, Lg = log(dd / dhat);
    o.E = -kappa * rr * rr * Lg;
    if (level < 1) return 1;
    const R b1 = -kappa * (R(2) * rr * Lg + rr * rr / dd);
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            R s = R(0);
            for (int z = 0; z < nb; ++z) s += R(coef[a][z]) * gz[3 * z + i];
            o.g[3 * a + i] = b1 * s;
        }
    if (level < 2) return 1;
    const R b2 = -kappa * (R(2) * Lg + R(4) * rr / dd - rr * rr / (dd * dd));
    const R il = R(1) / ell;
    // grad d in x (unscaled: grad_x d = grad_z~ d~), hess d in x = hess~ / ell
    R gx[12];
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            R s = R(0);
            for (int z = 0; z < nb; ++z) s += R(coef[a][z]) * gz[3 * z + i];
            gx[3 * a + i] = s;
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    R s = R(0);
                    for (int z = 0; z < nb; ++z)
                        for (int y = 0; y < nb; ++y) {
                            const int c = coef[a][z] * coef[b][y];
                            if (c) s += R(c) * Hz[(3 * z + i) * 9 + 3 * y + k];
                        }
                    o.H[(3 * a + i) * 12 + 3 * b + k] =
                        b2 * gx[3 * a + i] * gx[3 * b + k] + b1 * il * s;
                }
    return 1;
}

}  // namespace sx
