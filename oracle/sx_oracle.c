/*
 * sx_oracle.c -- plain FP64 CPU oracle for the energy-based time-integrator
 * hot path of "SymX: Energy-based Simulation from Symbolic Expressions".
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. The
 * product path (the CUDA library) never calls it, and the two share no
 * code: this file includes no header of the product and reimplements every
 * step from the paper in the most direct form, in double precision.
 *
 * What it computes (paper passages in brackets):
 *   - Stable Neo-Hookean tet4 energy, gradient, Hessian: element strain
 *     energy V_e psi(F_e) [§3.1, Eq. 7] with the Stable Neo-Hookean density
 *     [App. B, "Eq. 14 from Smith et al."]; derivatives by the chain rule
 *     through P = dpsi/dF and d2psi/dF2 and the constant 9x12 map vec(F) =
 *     B xhat built from Dm^-1 [App. A, tet4 shape functions].
 *   - The other tet4 densities of §6.1 / App. B (Neo-Hookean, St.
 *     Venant-Kirchhoff, fixed co-rotational and ARAP with lagged rotations)
 *     written as plain expressions of F and differentiated by second-order
 *     forward-mode arithmetic in the 12 stencil coordinates.
 *   - Quadratic hinge bending E = k_b/2 x^T Q x [§6.3, Eq. 13].
 *   - IPC log barrier E = -k (d - dhat)^2 ln(d/dhat) on the unsigned
 *     point-triangle distance [§6.4, Eq. 15], active only for d < dhat
 *     [§5.2 "Conditional evaluations", Eq. 9].
 *   - High-order (10- and 20-node) Lagrange tets with a quadrature sum
 *     [§6.2 Eq. 12, App. A shape functions].
 *   - Lagged IPC friction on point-triangle pairs [§6.4, friction
 *     potential] with its lag data (closest point, tangent basis, contact
 *     force) taken at the start of a step.
 *   - Per-element projection to positive semi-definiteness [§5.2
 *     "Projection to positive semi-definiteness", Algorithm 1 ProjectToPD]
 *     by cyclic Jacobi eigen-decomposition and eigenvalue clamping.
 *   - 3x3 block CRS pattern, element slot maps and ordered assembly of the
 *     global gradient and Hessian [§5.3, Eq. 11, Algorithm 1].
 *   - Inertia term of the backward-Euler incremental potential [§3, Eq. 2].
 *   - 3x3 block-Jacobi preconditioned CG [§7.2, linear solver paragraph].
 *   - Backward-Euler step by Newton's method with backtracking line search
 *     [§3, Eqs. 2-3; §5.1 three evaluation levels].
 *
 * Parity status: every function here is pinned by tests in tests/ against
 * closed forms, invariants, finite differences, library routines or brute
 * force (see the test files); none is "parity unpinned".
 *
 * Readings where the paper is silent or ambiguous are marked READING.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EDEGENERATE (-7)
#define ORC_ENOTCONV (-5)
#define ORC_ELINESEARCH (-9)
#define ORC_EINVALID_STATE (-6)

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major)                                      */
/* ------------------------------------------------------------------ */

/* Levi-Civita symbol for indices in {0,1,2}. */
static int levi(int i, int j, int k) { return (i - j) * (j - k) * (k - i) / 2; }

static double det3(const double A[9])
{
    double d = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                int e = levi(i, j, k);
                if (e) d += e * A[0 * 3 + i] * A[1 * 3 + j] * A[2 * 3 + k];
            }
    return d;
}

/* cof(F)_ij = 1/2 eps_imn eps_jpq F_mp F_nq  (= d det F / d F_ij). */
static void cofactor3(const double F[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n)
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) {
                            int e = levi(i, m, n) * levi(j, p, q);
                            if (e) s += e * F[m * 3 + p] * F[n * 3 + q];
                        }
            C[i * 3 + j] = 0.5 * s;
        }
}

/* inverse via cofactors: A^-1 = cof(A)^T / det A */
static void inv3(const double A[9], double Ai[9], double* detA)
{
    double C[9];
    cofactor3(A, C);
    double d = det3(A);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ai[i * 3 + j] = C[j * 3 + i] / d;
    if (detA) *detA = d;
}

/* ------------------------------------------------------------------ */
/* Stable Neo-Hookean material                                          */
/* ------------------------------------------------------------------ */

/* Lame parameters from Young's modulus and Poisson ratio (textbook
 * isotropic relations; the paper gives only E and nu, §6.1), then the
 * Stable Neo-Hookean re-parameterization of App. B. READING: the listing's
 * "4/3*mu" and "lambda + 5/6*lambda" are read as mu' = 4 mu / 3 and
 * lambda' = lambda + 5 mu / 6 (the form whose small-strain limit is linear
 * elasticity with mu, lambda; pinned by a test). literal != 0 keeps
 * mu' = mu, lambda' = lambda. */
void orc_snh_lame(int n, const double* E, const double* nu, int literal,
                  double* mu_s, double* lam_s)
{
    for (int e = 0; e < n; ++e) {
        double mu = E[e] / (2.0 * (1.0 + nu[e]));
        double lam = E[e] * nu[e] / ((1.0 + nu[e]) * (1.0 - 2.0 * nu[e]));
        if (literal) {
            mu_s[e] = mu;
            lam_s[e] = lam;
        } else {
            mu_s[e] = 4.0 * mu / 3.0;
            lam_s[e] = lam + 5.0 * mu / 6.0;
        }
    }
}

/* alpha of App. B: 1 + mu'/lambda' - mu'/(4 lambda'). READING: for
 * lambda' = 0 the volume term vanishes and alpha is taken as 1. */
static double snh_alpha(double mu, double lam)
{
    if (lam == 0.0) return 1.0;
    return 1.0 + mu / lam - mu / (4.0 * lam);
}

/* psi(F), P = dpsi/dF and d2psi/dF2 (9x9, vec index 3i+j) of the Stable
 * Neo-Hookean density psi = mu'/2 (Ic-3) + lambda'/2 (J-alpha)^2
 * - mu'/2 ln(Ic+1) [App. B]. READING: the energy is stored relative to
 * psi(I) so that the rest energy is zero; the constant changes no
 * derivative. psi(F) - psi(I) is written with the exact identities
 *   (J-alpha)^2 - (1-alpha)^2 = (J-1)(J+1-2 alpha),
 *   ln(Ic+1) - ln 4 = ln(1 + (Ic-3)/4),
 * and, with D = F - I, Ic - 3 = |D|^2 + 2 tr D and
 * J - 1 = det(I + D) - 1 = tr D + (sum of principal 2x2 minors of D) + det D,
 * so that no O(1) quantity is subtracted from another (otherwise the
 * energy carries an O(lambda' eps) absolute error per unit volume, far
 * above the last Newton decreases). */
static void snh_density(const double F[9], double mu, double lam,
                        double* psi, double P[9], double A[81])
{
    double alpha = snh_alpha(mu, lam);
    double D[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i * 3 + j] = F[i * 3 + j] - (i == j ? 1.0 : 0.0);
    double trD = D[0] + D[4] + D[8];
    double Ic3 = 2.0 * trD;
    for (int k = 0; k < 9; ++k) Ic3 += D[k] * D[k];
    double minors = (D[0] * D[4] - D[1] * D[3]) + (D[0] * D[8] - D[2] * D[6]) +
                    (D[4] * D[8] - D[5] * D[7]);
    double Jm1 = trD + minors + det3(D);
    double Ic = 3.0 + Ic3;
    double J = 1.0 + Jm1;
    double C[9];
    cofactor3(F, C);
    *psi = 0.5 * mu * Ic3 + 0.5 * lam * Jm1 * (J + 1.0 - 2.0 * alpha)
         - 0.5 * mu * log1p(0.25 * Ic3);
    if (P) {
        double a = mu * (1.0 - 1.0 / (Ic + 1.0));
        for (int k = 0; k < 9; ++k) P[k] = a * F[k] + lam * (J - alpha) * C[k];
    }
    if (A) {
        double a = mu * (1.0 - 1.0 / (Ic + 1.0));
        double b = 2.0 * mu / ((Ic + 1.0) * (Ic + 1.0));
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 9; ++c)
                A[r * 9 + c] = (r == c ? a : 0.0) + b * F[r] * F[c] + lam * C[r] * C[c];
        /* lambda'(J-alpha) d cof(F)_ij / d F_kl = eps_ikn eps_jlq F_nq */
        double s = lam * (J - alpha);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        double d = 0.0;
                        for (int n = 0; n < 3; ++n)
                            for (int q = 0; q < 3; ++q) {
                                int e = levi(i, k, n) * levi(j, l, q);
                                if (e) d += e * F[n * 3 + q];
                            }
                        A[(i * 3 + j) * 9 + (k * 3 + l)] += s * d;
                    }
    }
}

/* Rest quantities of a tet (App. A, linear tet4): Dm = [X1-X0, X2-X0,
 * X3-X0] (columns), its inverse, and V = det(Dm)/6. READING: the volume
 * must be positive; a non-positive det is reported as degenerate. */
int orc_tet_rest(int T, const double* X, const int* tets, double* Dminv, double* V)
{
    int bad = 0;
    for (int e = 0; e < T; ++e) {
        double Dm[9];
        const int* t = tets + 4 * e;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Dm[i * 3 + j] = X[3 * t[j + 1] + i] - X[3 * t[0] + i];
        double d;
        inv3(Dm, Dminv + 9 * e, &d);
        V[e] = d / 6.0;
        if (!(d > 0.0)) bad++;
    }
    return bad;
}

/* Lumped mass, READING: rho V_e / 4 to each vertex of every tet. */
void orc_lumped_mass(int N, int T, const int* tets, const double* V,
                     const double* rho, double* m)
{
    for (int n = 0; n < N; ++n) m[n] = 0.0;
    for (int e = 0; e < T; ++e)
        for (int a = 0; a < 4; ++a) m[tets[4 * e + a]] += rho[e] * V[e] / 4.0;
}

/* Gradient of the tet4 shape functions in rest coordinates: G (4x3) with
 * F_ij = sum_a x_{a,i} G_{a,j}; rows 1..3 are rows of Dm^-1 and row 0 is
 * minus their sum. The 9x12 map B has B[(3i+j),(3a+k)] = delta_ik G_aj. */
static void tet_B(const double Dminv[9], double B[9 * 12])
{
    double G[12];
    for (int j = 0; j < 3; ++j) {
        G[0 * 3 + j] = -(Dminv[0 * 3 + j] + Dminv[1 * 3 + j] + Dminv[2 * 3 + j]);
        for (int a = 1; a < 4; ++a) G[a * 3 + j] = Dminv[(a - 1) * 3 + j];
    }
    for (int r = 0; r < 9 * 12; ++r) B[r] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 4; ++a)
                B[(i * 3 + j) * 12 + (a * 3 + i)] = G[a * 3 + j];
}

/* One SNH tet: E = V psi(F), g = V B^T vec(P), H = V B^T (d2psi/dF2) B.
 * xe = 4 vertices x 3 coordinates. g or H may be NULL. */
void orc_snh_element(const double* xe, const double* Dminv, double V,
                     double mu, double lam, double* E, double* g, double* H)
{
    double B[9 * 12];
    tet_B(Dminv, B);
    double F[9];
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int c = 0; c < 12; ++c) s += B[r * 12 + c] * xe[c];
        F[r] = s;
    }
    double psi, P[9], A[81];
    snh_density(F, mu, lam, &psi, (g || H) ? P : NULL, H ? A : NULL);
    *E = V * psi;
    if (g)
        for (int c = 0; c < 12; ++c) {
            double s = 0.0;
            for (int r = 0; r < 9; ++r) s += B[r * 12 + c] * P[r];
            g[c] = V * s;
        }
    if (H) {
        double AB[9 * 12];
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 12; ++c) {
                double s = 0.0;
                for (int k = 0; k < 9; ++k) s += A[r * 9 + k] * B[k * 12 + c];
                AB[r * 12 + c] = s;
            }
        for (int r = 0; r < 12; ++r)
            for (int c = 0; c < 12; ++c) {
                double s = 0.0;
                for (int k = 0; k < 9; ++k) s += B[k * 12 + r] * AB[k * 12 + c];
                H[r * 12 + c] = V * s;
            }
    }
}

/* ------------------------------------------------------------------ */
/* Quadratic hinge bending (§6.3, Eq. 13)                               */
/* ------------------------------------------------------------------ */

/* READING: Q_e = c (q q^T kron I3) with q the cotangent weights of the flat
 * rest hinge and c = 3/(A0+A1) (Bergou et al., the cited construction);
 * the library takes q and c as per-stencil inputs. The oracle forms the
 * 12x12 Q and applies E = k/2 x^T Q x, g = k Q x, H = k Q literally. */
void orc_hinge_element(const double* xe, const double* q, double c, double kb,
                       double* E, double* g, double* H)
{
    double Q[144];
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
            for (int b = 0; b < 4; ++b)
                for (int j = 0; j < 3; ++j)
                    Q[(a * 3 + i) * 12 + (b * 3 + j)] = (i == j) ? c * q[a] * q[b] : 0.0;
    double Qx[12];
    for (int r = 0; r < 12; ++r) {
        double s = 0.0;
        for (int k = 0; k < 12; ++k) s += Q[r * 12 + k] * xe[k];
        Qx[r] = s;
    }
    double xQx = 0.0;
    for (int r = 0; r < 12; ++r) xQx += xe[r] * Qx[r];
    *E = 0.5 * kb * xQx;
    if (g) for (int r = 0; r < 12; ++r) g[r] = kb * Qx[r];
    if (H) for (int r = 0; r < 144; ++r) H[r] = kb * Q[r];
}

/* ------------------------------------------------------------------ */
/* Point-triangle barrier (§6.4, Eq. 15)                                */
/* ------------------------------------------------------------------ */

/* second-order forward-mode scalar: value, gradient and Hessian with
 * respect to the 12 stencil coordinates (p, t0, t1, t2). */
typedef struct { double v; double g[12]; double H[144]; } q2;

static void q2_const(q2* r, double v) { memset(r, 0, sizeof(*r)); r->v = v; }
static void q2_coord(q2* r, const double* xe, int node, int comp)
{
    q2_const(r, xe[3 * node + comp]);
    r->g[3 * node + comp] = 1.0;
}
static void q2_add(q2* r, const q2* a, const q2* b, double sb)
{
    q2 t;
    t.v = a->v + sb * b->v;
    for (int i = 0; i < 12; ++i) t.g[i] = a->g[i] + sb * b->g[i];
    for (int i = 0; i < 144; ++i) t.H[i] = a->H[i] + sb * b->H[i];
    *r = t;
}
/* product rule */
static void q2_mul(q2* r, const q2* a, const q2* b)
{
    q2 t;
    t.v = a->v * b->v;
    for (int i = 0; i < 12; ++i) t.g[i] = a->g[i] * b->v + a->v * b->g[i];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j)
            t.H[i * 12 + j] = a->H[i * 12 + j] * b->v + a->v * b->H[i * 12 + j]
                            + a->g[i] * b->g[j] + b->g[i] * a->g[j];
    *r = t;
}
/* chain rule for a scalar function f with derivatives f0, f1, f2 */
static void q2_apply(q2* r, const q2* a, double f0, double f1, double f2)
{
    q2 t;
    t.v = f0;
    for (int i = 0; i < 12; ++i) t.g[i] = f1 * a->g[i];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j)
            t.H[i * 12 + j] = f1 * a->H[i * 12 + j] + f2 * a->g[i] * a->g[j];
    *r = t;
}
static void q2_vec_sub(q2 r[3], const double* xe, int na, int nb)
{
    for (int k = 0; k < 3; ++k) {
        q2 a, b;
        q2_coord(&a, xe, na, k);
        q2_coord(&b, xe, nb, k);
        q2_add(&r[k], &a, &b, -1.0);
    }
}
static void q2_cross(q2 r[3], const q2 u[3], const q2 v[3])
{
    for (int k = 0; k < 3; ++k) {
        q2 s; q2_const(&s, 0.0);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                int e = levi(k, i, j);
                if (!e) continue;
                q2 t; q2_mul(&t, &u[i], &v[j]);
                q2_add(&s, &s, &t, (double)e);
            }
        r[k] = s;
    }
}
static void q2_dot(q2* r, const q2 u[3], const q2 v[3])
{
    q2 s; q2_const(&s, 0.0);
    for (int k = 0; k < 3; ++k) {
        q2 t; q2_mul(&t, &u[k], &v[k]);
        q2_add(&s, &s, &t, 1.0);
    }
    *r = s;
}

/* Closest-feature classification of point p against triangle (a,b,c) by
 * the textbook Voronoi-region tests (vertex regions first, then edges,
 * then the face), so that ties on a region boundary go to the
 * lower-dimensional feature. Returns 0,1,2 = vertex a,b,c; 3 = edge ab,
 * 4 = edge bc, 5 = edge ca; 6 = face. READING: the paper names the IPC
 * distance kernels without a formula (§6.4). */
int orc_pt_region(const double* xe)
{
    const double *p = xe, *a = xe + 3, *b = xe + 6, *c = xe + 9;
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int k = 0; k < 3; ++k) {
        ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k];
        ap[k] = p[k] - a[k]; bp[k] = p[k] - b[k]; cp[k] = p[k] - c[k];
    }
#define DOT(u, v) ((u)[0] * (v)[0] + (u)[1] * (v)[1] + (u)[2] * (v)[2])
    double d1 = DOT(ab, ap), d2 = DOT(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) return 0;
    double d3 = DOT(ab, bp), d4 = DOT(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) return 1;
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return 3;
    double d5 = DOT(ab, cp), d6 = DOT(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) return 2;
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return 5;
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) return 4;
    return 6;
#undef DOT
}

/* Squared distance s = |r|^2 / w of the active feature, with gradient and
 * Hessian, through the quotient s w = sum r_k^2 differentiated twice:
 * vertex v: r = p - v, w = 1; edge (u,v): r = (p-u) x (v-u), w = |v-u|^2;
 * face: r = (p-a).((b-a)x(c-a)), w = |(b-a)x(c-a)|^2. */
static void pt_sqdist(const double* xe, int region, q2* s)
{
    q2 num, w;
    if (region <= 2) {
        q2 r[3];
        q2_vec_sub(r, xe, 0, 1 + region);
        q2_dot(&num, r, r);
        q2_const(&w, 1.0);
    } else if (region <= 5) {
        int u = (region == 3) ? 1 : (region == 4 ? 2 : 3);
        int v = (region == 3) ? 2 : (region == 4 ? 3 : 1);
        q2 e[3], d[3], r[3];
        q2_vec_sub(e, xe, 0, u);
        q2_vec_sub(d, xe, v, u);
        q2_cross(r, e, d);
        q2_dot(&num, r, r);
        q2_dot(&w, d, d);
    } else {
        q2 e[3], e1[3], e2[3], N[3], u;
        q2_vec_sub(e, xe, 0, 1);
        q2_vec_sub(e1, xe, 2, 1);
        q2_vec_sub(e2, xe, 3, 1);
        q2_cross(N, e1, e2);
        q2_dot(&u, e, N);
        q2_mul(&num, &u, &u);
        q2_dot(&w, N, N);
    }
    /* s = num / w: s w = num  =>  grad s = (grad num - s grad w)/w,
     * hess s = (hess num - grad s grad w^T - grad w grad s^T - s hess w)/w */
    q2 t;
    t.v = num.v / w.v;
    for (int i = 0; i < 12; ++i) t.g[i] = (num.g[i] - t.v * w.g[i]) / w.v;
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j)
            t.H[i * 12 + j] = (num.H[i * 12 + j] - t.g[i] * w.g[j] - w.g[i] * t.g[j]
                               - t.v * w.H[i * 12 + j]) / w.v;
    *s = t;
}

/* Unsigned point-triangle distance. */
double orc_pt_distance(const double* xe)
{
    q2 s;
    pt_sqdist(xe, orc_pt_region(xe), &s);
    return sqrt(s.v);
}

/* b(d) = -kappa (d-dhat)^2 ln(d/dhat) and its first two derivatives. */
void orc_barrier_1d(double d, double dhat, double kappa, double* b, double* b1, double* b2)
{
    double r = d - dhat, L = log(d / dhat);
    *b = -kappa * r * r * L;
    *b1 = -kappa * (2.0 * r * L + r * r / d);
    *b2 = -kappa * (2.0 * L + 4.0 * r / d - r * r / (d * d));
}

/* Barrier element: returns 1 when active (0 < d < dhat), 0 when inactive
 * (E, g, H zero: the element contributes nothing, Eq. 9), -1 for d <= 0
 * (an intersecting state the barrier does not admit). */
int orc_barrier_element(const double* xe, double dhat, double kappa,
                        double* E, double* g, double* H)
{
    q2 s;
    int region = orc_pt_region(xe);
    pt_sqdist(xe, region, &s);
    *E = 0.0;
    if (g) memset(g, 0, 12 * sizeof(double));
    if (H) memset(H, 0, 144 * sizeof(double));
    if (!(s.v > 0.0)) return -1;
    double d0 = sqrt(s.v);
    if (!(d0 < dhat)) return 0;
    /* d = sqrt(s) */
    q2 d;
    q2_apply(&d, &s, d0, 0.5 / d0, -0.25 / (s.v * d0));
    double b, b1, b2;
    orc_barrier_1d(d0, dhat, kappa, &b, &b1, &b2);
    q2 e;
    q2_apply(&e, &d, b, b1, b2);
    *E = e.v;
    if (g) memcpy(g, e.g, sizeof(e.g));
    if (H) memcpy(H, e.H, sizeof(e.H));
    return 1;
}

/* ------------------------------------------------------------------ */
/* Projection to PSD (§5.2; Algorithm 1 ProjectToPD)                    */
/* ------------------------------------------------------------------ */

/* Cyclic Jacobi (textbook symmetric Schur rotations) until the
 * off-diagonal norm is <= 1e-15 ||A||_F (at most 50 sweeps), then
 * A <- sum_i max(lambda_i, 0) v_i v_i^T. READING: the paper says
 * "positive semi-definiteness" (§5.2) and "ProjectToPD" (Algorithm 1);
 * clamping at 0 is taken. Returns the sweeps used or -1 if the sweep limit
 * was reached. n <= 12. */
int orc_clamp_psd(int n, double* A)
{
    double V[144], W[144];
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
    fro = sqrt(fro);
    if (fro == 0.0) return 0;
    for (int i = 0; i < n * n; ++i) W[i] = A[i];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    int sweep, ok = 0;
    for (sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += W[i * n + j] * W[i * n + j];
        if (sqrt(off) <= 1e-15 * fro) { ok = 1; break; }
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = W[p * n + q];
                if (apq == 0.0) continue;
                double tau = (W[q * n + q] - W[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = W[k * n + p], akq = W[k * n + q];
                    W[k * n + p] = c * akp - s * akq;
                    W[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = W[p * n + k], aqk = W[q * n + k];
                    W[p * n + k] = c * apk - s * aqk;
                    W[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                double lk = W[k * n + k];
                if (lk > 0.0) s += lk * V[i * n + k] * V[j * n + k];
            }
            A[i * n + j] = s;
        }
    return ok ? sweep : -1;
}

/* eigenvalues (ascending order not guaranteed) by the same Jacobi
 * iteration, for tests */
int orc_sym_eigvals(int n, const double* A, double* lam)
{
    double W[144], fro = 0.0;
    for (int i = 0; i < n * n; ++i) { W[i] = A[i]; fro += A[i] * A[i]; }
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 50 && fro > 0.0; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += W[i * n + j] * W[i * n + j];
        if (sqrt(off) <= 1e-15 * fro) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = W[p * n + q];
                if (apq == 0.0) continue;
                double tau = (W[q * n + q] - W[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = W[k * n + p], akq = W[k * n + q];
                    W[k * n + p] = c * akp - s * akq;
                    W[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = W[p * n + k], aqk = W[q * n + k];
                    W[p * n + k] = c * apk - s * aqk;
                    W[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = W[i * n + i];
    return sweep;
}

/* ------------------------------------------------------------------ */
/* Batched element evaluation (the parallel element loop of Alg. 1)     */
/* ------------------------------------------------------------------ */

static void gather4(const double* x, const int* t, double xe[12])
{
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) xe[3 * a + i] = x[3 * t[a] + i];
}

/* The SNH element Hessian with the material Hessian d2psi/dF2 projected to
 * positive semi-definiteness before the chain rule: H = V B^T proj(d2psi/dF2) B
 * with proj the eigenvalue clamp at zero of the 9x9 (§5.2's projection taken
 * on the F-space Hessian rather than on the 12x12 element Hessian; the
 * survey's "next" row of an analytic projection). The 9x9 is clamped by the
 * same cyclic Jacobi as the 12x12. E and g are those of orc_snh_element. */
void orc_snh_element_fproj(const double* xe, const double* Dminv, double V,
                           double mu, double lam, double* E, double* g, double* H)
{
    double B[9 * 12];
    tet_B(Dminv, B);
    double F[9];
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int c = 0; c < 12; ++c) s += B[r * 12 + c] * xe[c];
        F[r] = s;
    }
    double psi, P[9], A[81];
    snh_density(F, mu, lam, &psi, P, A);
    *E = V * psi;
    if (g)
        for (int c = 0; c < 12; ++c) {
            double s = 0.0;
            for (int r = 0; r < 9; ++r) s += B[r * 12 + c] * P[r];
            g[c] = V * s;
        }
    if (H) {
        orc_clamp_psd(9, A);
        double AB[9 * 12];
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 12; ++c) {
                double s = 0.0;
                for (int k = 0; k < 9; ++k) s += A[r * 9 + k] * B[k * 12 + c];
                AB[r * 12 + c] = s;
            }
        for (int r = 0; r < 12; ++r)
            for (int c = 0; c < 12; ++c) {
                double s = 0.0;
                for (int k = 0; k < 9; ++k) s += B[k * 12 + r] * AB[k * 12 + c];
                H[r * 12 + c] = V * s;
            }
    }
}

/* d2psi/dF2 (9x9, vec index 3i+j) of one SNH tet at its deformation
 * gradient, for checks of the F-space projection. */
void orc_snh_dPdF(const double* xe, const double* Dminv, double mu, double lam, double* A)
{
    double B[9 * 12];
    tet_B(Dminv, B);
    double F[9];
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int c = 0; c < 12; ++c) s += B[r * 12 + c] * xe[c];
        F[r] = s;
    }
    double psi, P[9];
    snh_density(F, mu, lam, &psi, P, A);
}

/* level: 0 = E, 1 = E+g, 2 = E+g+H. H_e is 144 per element (row-major).
 * project: 0 none, 1 clamp of the 12x12 H, 2 clamp of d2psi/dF2. */
void orc_snh_batch(int T, const double* x, const int* tets, const double* Dminv,
                   const double* V, const double* mu, const double* lam,
                   int level, int project, double* E_e, double* g_e, double* H_e)
{
#pragma omp parallel for schedule(static)
    for (int e = 0; e < T; ++e) {
        double xe[12];
        gather4(x, tets + 4 * e, xe);
        if (level >= 2 && project == 2) {
            orc_snh_element_fproj(xe, Dminv + 9 * e, V[e], mu[e], lam[e], E_e + e,
                                  g_e + 12 * (size_t)e, H_e + 144 * (size_t)e);
            continue;
        }
        orc_snh_element(xe, Dminv + 9 * e, V[e], mu[e], lam[e], E_e + e,
                        level >= 1 ? g_e + 12 * (size_t)e : NULL,
                        level >= 2 ? H_e + 144 * (size_t)e : NULL);
        if (level >= 2 && project) orc_clamp_psd(12, H_e + 144 * (size_t)e);
    }
}

void orc_hinge_batch(int S, const double* x, const int* st, const double* q,
                     const double* c, double kb, int level,
                     double* E_e, double* g_e, double* H_e)
{
#pragma omp parallel for schedule(static)
    for (int e = 0; e < S; ++e) {
        double xe[12];
        gather4(x, st + 4 * e, xe);
        orc_hinge_element(xe, q + 4 * e, c[e], kb, E_e + e,
                          level >= 1 ? g_e + 12 * (size_t)e : NULL,
                          level >= 2 ? H_e + 144 * (size_t)e : NULL);
    }
}

/* returns the number of pairs with d <= 0 (invalid state) */
int orc_barrier_batch(int P, const double* x, const int* pairs, double dhat,
                      double kappa, int level, int project,
                      double* E_e, double* g_e, double* H_e, int* active)
{
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int e = 0; e < P; ++e) {
        double xe[12], gl[12], Hl[144];
        gather4(x, pairs + 4 * e, xe);
        int st = orc_barrier_element(xe, dhat, kappa, E_e + e, gl, Hl);
        if (st < 0) bad++;
        if (active) active[e] = st;
        if (level >= 1) memcpy(g_e + 12 * (size_t)e, gl, sizeof(gl));
        if (level >= 2) {
            if (project && st == 1) orc_clamp_psd(12, Hl);
            memcpy(H_e + 144 * (size_t)e, Hl, sizeof(Hl));
        }
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Other tet4 densities (§6.1 "Non-Linear Material Models", App. B):    */
/* Neo-Hookean, St. Venant-Kirchhoff, fixed co-rotational and ARAP with */
/* a volume term, the two co-rotational ones with a lagged rotation R   */
/* ------------------------------------------------------------------ */

#define ORC_MODEL_SNH 0
#define ORC_MODEL_NH 1
#define ORC_MODEL_STVK 2
#define ORC_MODEL_COROT 3
#define ORC_MODEL_ARAP 4

/* u - ln(1 + u) without cancellation: for |u| < 1/16 the alternating
 * series sum_{k >= 2} (-1)^k u^k / k, up to k = 20 (the tail is below
 * 1e-20 of the sum there); otherwise the direct difference. */
static double u_minus_log1p(double u)
{
    if (fabs(u) < 0.0625) {
        double s = 0.0, p = u * u;
        for (int k = 2; k <= 20; ++k) {
            s += ((k & 1) ? -p : p) / (double)k;
            p *= u;
        }
        return s;
    }
    return u - log1p(u);
}

/* F_ij = sum_a x_{a,i} G_{a,j} as second-order jets in the 12 stencil
 * coordinates (F is linear in them: constant gradient, zero Hessian). */
static void tet_F_jets(const double* xe, const double Dminv[9], q2 F[9])
{
    double B[9 * 12];
    tet_B(Dminv, B);
    for (int r = 0; r < 9; ++r) {
        q2_const(&F[r], 0.0);
        for (int c = 0; c < 12; ++c) {
            F[r].v += B[r * 12 + c] * xe[c];
            F[r].g[c] = B[r * 12 + c];
        }
    }
}

static void q2_sq_sum(q2* r, const q2* a, int n)
{
    q2 s;
    q2_const(&s, 0.0);
    for (int k = 0; k < n; ++k) {
        q2 t;
        q2_mul(&t, &a[k], &a[k]);
        q2_add(&s, &s, &t, 1.0);
    }
    *r = s;
}

/* J - 1 = det(I + D) - 1 = tr D + (sum of principal 2x2 minors of D) + det D
 * for D = F - I, as a jet (no O(1) quantity is subtracted). */
static void q2_jm1(q2* r, const q2 D[9])
{
    q2 s, t, u;
    q2_add(&s, &D[0], &D[4], 1.0);
    q2_add(&s, &s, &D[8], 1.0);
    static const int mi[3][4] = {{0, 4, 1, 3}, {0, 8, 2, 6}, {4, 8, 5, 7}};
    for (int m = 0; m < 3; ++m) {
        q2_mul(&t, &D[mi[m][0]], &D[mi[m][1]]);
        q2_mul(&u, &D[mi[m][2]], &D[mi[m][3]]);
        q2_add(&t, &t, &u, -1.0);
        q2_add(&s, &s, &t, 1.0);
    }
    /* det D by the permutation sum eps_ijk D_0i D_1j D_2k */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                int e = levi(i, j, k);
                if (!e) continue;
                q2_mul(&t, &D[0 * 3 + i], &D[1 * 3 + j]);
                q2_mul(&t, &t, &D[2 * 3 + k]);
                q2_add(&s, &s, &t, (double)e);
            }
    *r = s;
}

/* psi of a non-SNH model as a jet in the stencil coordinates. Returns 1
 * for a state where the density is undefined (Neo-Hookean with J <= 0).
 * Each density is written as its definition with F = I + D:
 *   NH    mu/2 (Ic - 3) - mu ln J + lambda/2 ln^2 J (Smith et al. Eq. 5; the
 *         text form of §3.1 prints +mu ln J, READING: the minus sign, the
 *         only one for which the rest state is stress-free), expanded as
 *         mu/2 |D|^2 - mu (minors + det D) + mu (u - ln(1+u))
 *         + lambda/2 ln^2(1+u), u = J - 1, which is the same function;
 *   StVK  mu |E|^2 + lambda/2 tr(E)^2, E = (F^T F - I)/2 = (D + D^T + D^T D)/2;
 *   COROT mu |F - R|^2 + lambda/2 (J - 1)^2;
 *   ARAP  mu/2 (Ic - 2 tr(F^T R) + 3) + lambda/2 (J - 1)^2, written as
 *         mu/2 |F - R|^2 (equal for a rotation R, |R|^2 = 3).
 * R (row-major) is constant: the rotation is lagged (held for the time
 * step), so no derivative of R enters. */
static int tet_psi_jet(int model, const q2 F[9], const double R[9], double mu, double lam,
                       q2* psi)
{
    q2 D[9];
    for (int k = 0; k < 9; ++k) {
        D[k] = F[k];
        if (k % 4 == 0) D[k].v -= 1.0;
    }
    q2 t, u;
    if (model == ORC_MODEL_NH) {
        q2 jm1;
        q2_jm1(&jm1, D);
        if (!(jm1.v > -1.0)) return 1;
        q2_sq_sum(psi, D, 9);
        q2_apply(psi, psi, 0.5 * mu * psi->v, 0.5 * mu, 0.0);
        /* minors + det D = (J - 1) - tr D */
        q2_add(&t, &jm1, &D[0], -1.0);
        q2_add(&t, &t, &D[4], -1.0);
        q2_add(&t, &t, &D[8], -1.0);
        q2_add(psi, psi, &t, -mu);
        const double w = jm1.v, ip = 1.0 / (1.0 + w);
        /* f(u) = u - ln(1+u): f' = u/(1+u), f'' = 1/(1+u)^2 */
        q2_apply(&t, &jm1, u_minus_log1p(w), w * ip, ip * ip);
        q2_add(psi, psi, &t, mu);
        /* ln(1+u): derivatives 1/(1+u), -1/(1+u)^2; then its square */
        q2_apply(&u, &jm1, log1p(w), ip, -ip * ip);
        q2_mul(&t, &u, &u);
        q2_add(psi, psi, &t, 0.5 * lam);
        return 0;
    }
    if (model == ORC_MODEL_STVK) {
        q2 E[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                q2 s;
                q2_add(&s, &D[i * 3 + j], &D[j * 3 + i], 1.0);
                for (int m = 0; m < 3; ++m) {
                    q2_mul(&t, &D[m * 3 + i], &D[m * 3 + j]);
                    q2_add(&s, &s, &t, 1.0);
                }
                q2_apply(&E[i * 3 + j], &s, 0.5 * s.v, 0.5, 0.0);
            }
        q2_sq_sum(psi, E, 9);
        q2_apply(psi, psi, mu * psi->v, mu, 0.0);
        q2_add(&t, &E[0], &E[4], 1.0);
        q2_add(&t, &t, &E[8], 1.0);
        q2_mul(&u, &t, &t);
        q2_add(psi, psi, &u, 0.5 * lam);
        return 0;
    }
    /* COROT / ARAP */
    q2 FR[9];
    for (int k = 0; k < 9; ++k) {
        FR[k] = F[k];
        FR[k].v -= R[k];
    }
    q2_sq_sum(psi, FR, 9);
    const double c = (model == ORC_MODEL_COROT) ? mu : 0.5 * mu;
    q2_apply(psi, psi, c * psi->v, c, 0.0);
    q2 jm1;
    q2_jm1(&jm1, D);
    q2_mul(&t, &jm1, &jm1);
    q2_add(psi, psi, &t, 0.5 * lam);
    return 0;
}

/* One tet of any model: E = V psi, g = V dpsi/dx, H = V d2psi/dx2 (the
 * SNH model goes through orc_snh_element). R: row-major 3x3, used by
 * COROT and ARAP only (may be NULL otherwise). Returns 1 for an invalid
 * state (NH with J <= 0; E, g and H are then zero). */
int orc_tet_element(int model, const double* xe, const double* Dminv, double V,
                    double mu, double lam, const double* R, double* E, double* g, double* H)
{
    if (model == ORC_MODEL_SNH) {
        orc_snh_element(xe, Dminv, V, mu, lam, E, g, H);
        return 0;
    }
    q2 F[9], psi;
    tet_F_jets(xe, Dminv, F);
    static const double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (tet_psi_jet(model, F, R ? R : I3, mu, lam, &psi)) {
        *E = 0.0;
        if (g) memset(g, 0, 12 * sizeof(double));
        if (H) memset(H, 0, 144 * sizeof(double));
        return 1;
    }
    *E = V * psi.v;
    if (g)
        for (int c = 0; c < 12; ++c) g[c] = V * psi.g[c];
    if (H)
        for (int c = 0; c < 144; ++c) H[c] = V * psi.H[c];
    return 0;
}

/* Batch of one model. project: 0 none, 1 clamp of the 12x12, 2 clamp of
 * d2psi/dF2 for SNH (READING: other models have no F-space projection
 * and take the 12x12 clamp). R: 9 per tet (COROT / ARAP). Returns the
 * number of tets in an invalid state. */
int orc_tet_batch(int model, int T, const double* x, const int* tets, const double* Dminv,
                  const double* V, const double* mu, const double* lam, const double* R,
                  int level, int project, double* E_e, double* g_e, double* H_e)
{
    if (model == ORC_MODEL_SNH) {
        orc_snh_batch(T, x, tets, Dminv, V, mu, lam, level, project, E_e, g_e, H_e);
        return 0;
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int e = 0; e < T; ++e) {
        double xe[12];
        gather4(x, tets + 4 * e, xe);
        bad += orc_tet_element(model, xe, Dminv + 9 * e, V[e], mu[e], lam[e],
                               R ? R + 9 * (size_t)e : NULL, E_e + e,
                               level >= 1 ? g_e + 12 * (size_t)e : NULL,
                               level >= 2 ? H_e + 144 * (size_t)e : NULL);
        if (level >= 2 && project) orc_clamp_psd(12, H_e + 144 * (size_t)e);
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Lagged IPC friction on point-triangle pairs (§6.4, friction          */
/* potential)                                                           */
/* ------------------------------------------------------------------ */

/* Closest point of triangle (a, b, c) to p as barycentric weights, from
 * the Voronoi region of orc_pt_region: a vertex gets weight 1, an edge
 * (u, v) the clamped projection parameter t (weights 1 - t, t), the face
 * the barycentrics of the plane projection. */
static void pt_closest_weights(const double* xe, double beta[3])
{
    const double *p = xe, *t[3] = {xe + 3, xe + 6, xe + 9};
    int reg = orc_pt_region(xe);
    beta[0] = beta[1] = beta[2] = 0.0;
    if (reg <= 2) {
        beta[reg] = 1.0;
        return;
    }
    if (reg <= 5) {
        int u = reg - 3, v = (reg - 3 + 1) % 3;
        double num = 0.0, den = 0.0;
        for (int k = 0; k < 3; ++k) {
            double e = t[v][k] - t[u][k];
            num += (p[k] - t[u][k]) * e;
            den += e * e;
        }
        double tt = den > 0.0 ? num / den : 0.0;
        if (tt < 0.0) tt = 0.0;
        if (tt > 1.0) tt = 1.0;
        beta[u] = 1.0 - tt;
        beta[v] = tt;
        return;
    }
    double ab[3], ac[3], ap[3];
    for (int k = 0; k < 3; ++k) {
        ab[k] = t[1][k] - t[0][k];
        ac[k] = t[2][k] - t[0][k];
        ap[k] = p[k] - t[0][k];
    }
    double d00 = 0, d01 = 0, d11 = 0, d20 = 0, d21 = 0;
    for (int k = 0; k < 3; ++k) {
        d00 += ab[k] * ab[k]; d01 += ab[k] * ac[k]; d11 += ac[k] * ac[k];
        d20 += ap[k] * ab[k]; d21 += ap[k] * ac[k];
    }
    double den = d00 * d11 - d01 * d01;
    double v = (d11 * d20 - d01 * d21) / den, w = (d00 * d21 - d01 * d20) / den;
    beta[0] = 1.0 - v - w;
    beta[1] = v;
    beta[2] = w;
}

/* Lagged contact data of one pair at the state xe (p, t0, t1, t2), held
 * for a time step like IPC's lagged friction. READINGS (the paper gives
 * the potential, not its lagged inputs): the contact point is the closest
 * point c of the triangle; f_n = -b'(d) is the magnitude of the barrier's
 * contact force at d = |p - c| (zero outside 0 < d < dhat); T (2x3, rows)
 * is an orthonormal basis of the plane normal to p - c (any basis gives
 * the same potential). out: beta[3], T[6], fn, dxt[3] = p - c. */
void orc_friction_lag(const double* xe, double dhat, double kappa, double* beta, double* T,
                      double* fn, double* dxt)
{
    pt_closest_weights(xe, beta);
    double r[3], d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double c = beta[0] * xe[3 + k] + beta[1] * xe[6 + k] + beta[2] * xe[9 + k];
        r[k] = xe[k] - c;
        dxt[k] = r[k];
        d2 += r[k] * r[k];
    }
    double d = sqrt(d2);
    *fn = 0.0;
    if (d > 0.0 && d < dhat) {
        double b, b1, b2;
        orc_barrier_1d(d, dhat, kappa, &b, &b1, &b2);
        *fn = -b1;
    }
    double n[3] = {0.0, 0.0, 1.0};
    if (d > 0.0)
        for (int k = 0; k < 3; ++k) n[k] = r[k] / d;
    /* first tangent: n x (the axis least aligned with n), normalized */
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (fabs(n[k]) < fabs(n[ax])) ax = k;
    double e[3] = {0.0, 0.0, 0.0};
    e[ax] = 1.0;
    double t1[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
    double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int k = 0; k < 3; ++k) t1[k] /= l;
    double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
    for (int k = 0; k < 3; ++k) {
        T[k] = t1[k];
        T[3 + k] = t2[k];
    }
}

/* f0(s) = dt f(s/dt) with the friction profile of §6.4:
 * f(y) = -y^3/(3 yh^2) + y^2/yh + yh/3 for y <= yh, y otherwise; and its
 * first two derivatives in s. */
static void friction_f0(double s, double yh, double dt, double* f, double* f1, double* f2)
{
    double y = s / dt;
    if (y <= yh) {
        *f = dt * (-y * y * y / (3.0 * yh * yh) + y * y / yh + yh / 3.0);
        *f1 = -y * y / (yh * yh) + 2.0 * y / yh;
        *f2 = (-2.0 * y / (yh * yh) + 2.0 / yh) / dt;
    } else {
        *f = dt * y;
        *f1 = 1.0;
        *f2 = 0.0;
    }
}

/* One friction stencil: E = mu fn f0(s), s = |T (dx - dxt)|, with
 * dx = p - sum_i beta_i t_i the current separation at the lagged contact
 * point, so T (dx - dxt) / dt is the tangential relative velocity y of
 * §6.4 over the step. READING: the potential is taken as dt mu fn f(y)
 * (= mu fn f0(s)), the incremental potential of the friction force, whose
 * sliding force is mu fn (IPC's lagged friction potential with threshold
 * yh dt). At s = 0 the derivatives are the limits (g = 0,
 * H = mu fn 2/(yh dt) J^T J). */
void orc_friction_element(const double* xe, const double* beta, const double* T, double fn,
                          const double* dxt, double mu, double yhat, double dt,
                          double* E, double* g, double* H)
{
    q2 u[2];
    for (int j = 0; j < 2; ++j) {
        q2_const(&u[j], 0.0);
        for (int k = 0; k < 3; ++k) {
            double w = xe[k] - beta[0] * xe[3 + k] - beta[1] * xe[6 + k] - beta[2] * xe[9 + k]
                     - dxt[k];
            u[j].v += T[3 * j + k] * w;
            u[j].g[k] += T[3 * j + k];
            for (int i = 0; i < 3; ++i) u[j].g[3 * (i + 1) + k] -= T[3 * j + k] * beta[i];
        }
    }
    q2 s2, t;
    q2_mul(&s2, &u[0], &u[0]);
    q2_mul(&t, &u[1], &u[1]);
    q2_add(&s2, &s2, &t, 1.0);
    const double k = mu * fn;
    if (s2.v > 0.0) {
        double sv = sqrt(s2.v), f, f1, f2;
        q2 s;
        q2_apply(&s, &s2, sv, 0.5 / sv, -0.25 / (sv * sv * sv));
        friction_f0(sv, yhat, dt, &f, &f1, &f2);
        q2_apply(&t, &s, f, f1, f2);
        *E = k * t.v;
        if (g) for (int c = 0; c < 12; ++c) g[c] = k * t.g[c];
        if (H) for (int c = 0; c < 144; ++c) H[c] = k * t.H[c];
        return;
    }
    *E = k * dt * yhat / 3.0;
    if (g) memset(g, 0, 12 * sizeof(double));
    if (H) {
        /* J^T J with J the (constant) gradients of u */
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b)
                H[a * 12 + b] = k * 2.0 / (yhat * dt) *
                                (u[0].g[a] * u[0].g[b] + u[1].g[a] * u[1].g[b]);
    }
}

void orc_friction_lag_batch(int P, const double* x, const int* pairs, double dhat, double kappa,
                            double* beta, double* T, double* fn, double* dxt)
{
#pragma omp parallel for schedule(static)
    for (int e = 0; e < P; ++e) {
        double xe[12];
        gather4(x, pairs + 4 * e, xe);
        orc_friction_lag(xe, dhat, kappa, beta + 3 * (size_t)e, T + 6 * (size_t)e, fn + e,
                         dxt + 3 * (size_t)e);
    }
}

void orc_friction_batch(int P, const double* x, const int* pairs, const double* beta,
                        const double* T, const double* fn, const double* dxt, double mu,
                        double yhat, double dt, int level, double* E_e, double* g_e, double* H_e)
{
#pragma omp parallel for schedule(static)
    for (int e = 0; e < P; ++e) {
        double xe[12];
        gather4(x, pairs + 4 * e, xe);
        orc_friction_element(xe, beta + 3 * (size_t)e, T + 6 * (size_t)e, fn[e],
                             dxt + 3 * (size_t)e, mu, yhat, dt, E_e + e,
                             level >= 1 ? g_e + 12 * (size_t)e : NULL,
                             level >= 2 ? H_e + 144 * (size_t)e : NULL);
    }
}

/* ------------------------------------------------------------------ */
/* High-order Lagrange tets with a quadrature sum (§6.2 "High-order      */
/* Lagrangian finite elements", Eq. 12; App. A shape functions;       */
/* §5 fixed-value summation)                                            */
/* ------------------------------------------------------------------ */

/* Local node order. Barycentric L = (1 - xi0 - xi1 - xi2, xi0, xi1, xi2).
 * tet4: the vertices. tet10 (App. A): the vertices, then one node per edge
 * in the order 01, 12, 20, 03, 13, 23. tet20 (READING: the paper shows no
 * cubic listing; the standard cubic Lagrange tet): the vertices; two nodes
 * per edge in the same edge order, first the one nearer the edge's first
 * vertex; one node per face in the order 012, 013, 123, 023. */
static const int ORC_EDGES[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
static const int ORC_FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

/* Shape functions N (K) and their reference gradients dN (K x 3) at xi. */
void orc_tetho_shape(int K, const double* xi, double* N, double* dN)
{
    double L[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
    static const double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    /* each N as a function of L with its partials dN/dL, then the chain rule */
    double dNL[20][4];
    memset(dNL, 0, sizeof(dNL));
    int a = 0;
    if (K == 4) {
        for (int v = 0; v < 4; ++v, ++a) { N[a] = L[v]; dNL[a][v] = 1.0; }
    } else if (K == 10) {
        for (int v = 0; v < 4; ++v, ++a) {
            N[a] = L[v] * (2.0 * L[v] - 1.0);
            dNL[a][v] = 4.0 * L[v] - 1.0;
        }
        for (int e = 0; e < 6; ++e, ++a) {
            int i = ORC_EDGES[e][0], j = ORC_EDGES[e][1];
            N[a] = 4.0 * L[i] * L[j];
            dNL[a][i] = 4.0 * L[j];
            dNL[a][j] = 4.0 * L[i];
        }
    } else {
        for (int v = 0; v < 4; ++v, ++a) {
            double l = L[v];
            N[a] = 0.5 * l * (3.0 * l - 1.0) * (3.0 * l - 2.0);
            dNL[a][v] = 0.5 * (27.0 * l * l - 18.0 * l + 2.0);
        }
        for (int e = 0; e < 6; ++e)
            for (int side = 0; side < 2; ++side, ++a) {
                int i = ORC_EDGES[e][side], j = ORC_EDGES[e][1 - side];
                /* node nearer i: 9/2 L_i L_j (3 L_i - 1) */
                N[a] = 4.5 * L[i] * L[j] * (3.0 * L[i] - 1.0);
                dNL[a][i] = 4.5 * L[j] * (6.0 * L[i] - 1.0);
                dNL[a][j] = 4.5 * L[i] * (3.0 * L[i] - 1.0);
            }
        for (int f = 0; f < 4; ++f, ++a) {
            int i = ORC_FACES[f][0], j = ORC_FACES[f][1], k = ORC_FACES[f][2];
            N[a] = 27.0 * L[i] * L[j] * L[k];
            dNL[a][i] = 27.0 * L[j] * L[k];
            dNL[a][j] = 27.0 * L[i] * L[k];
            dNL[a][k] = 27.0 * L[i] * L[j];
        }
    }
    for (int b = 0; b < K; ++b)
        for (int m = 0; m < 3; ++m) {
            double sdn = 0.0;
            for (int v = 0; v < 4; ++v) sdn += dNL[b][v] * dL[v][m];
            dN[3 * b + m] = sdn;
        }
}

/* One SNH element of K nodes: E = sum_q w_q det(J0_q) psi(F_q) with
 * J0 = sum_a X_a dN_a^T, F = (sum_a x_a dN_a^T) J0^-1 at the quadrature
 * point xi_q (Eq. 12); g and H by the chain rule through the 9 x 3K
 * map of each point. rule: nq x (w, xi0, xi1, xi2). project != 0 clamps
 * d2psi/dF2 at every point (READING: the PSD projection of high-order
 * elements is taken per quadrature point in F-space; the sum of PSD terms
 * is PSD). Returns 1 if some det(J0_q) <= 0. */
int orc_tetho_element(int K, int nq, const double* rule, const double* Xe, const double* xe,
                      double mu, double lam, int project, double* E, double* g, double* H)
{
    int n3 = 3 * K, bad = 0;
    double N[20], dN[60], B[9 * 60];
    *E = 0.0;
    if (g) memset(g, 0, n3 * sizeof(double));
    if (H) memset(H, 0, (size_t)n3 * n3 * sizeof(double));
    for (int q = 0; q < nq; ++q) {
        const double w = rule[4 * q];
        orc_tetho_shape(K, rule + 4 * q + 1, N, dN);
        double J0[9] = {0}, Ds[9] = {0}, J0i[9], det;
        for (int a = 0; a < K; ++a)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    J0[3 * i + j] += Xe[3 * a + i] * dN[3 * a + j];
                    Ds[3 * i + j] += xe[3 * a + i] * dN[3 * a + j];
                }
        inv3(J0, J0i, &det);
        if (!(det > 0.0)) bad = 1;
        double F[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double sf = 0.0;
                for (int m = 0; m < 3; ++m) sf += Ds[3 * i + m] * J0i[3 * m + j];
                F[3 * i + j] = sf;
            }
        /* B[(3i+j), (3a+k)] = delta_ik G_aj, G_a = J0^-T dN_a */
        memset(B, 0, sizeof(double) * 9 * n3);
        for (int a = 0; a < K; ++a)
            for (int j = 0; j < 3; ++j) {
                double G = 0.0;
                for (int m = 0; m < 3; ++m) G += dN[3 * a + m] * J0i[3 * m + j];
                for (int i = 0; i < 3; ++i) B[(3 * i + j) * n3 + 3 * a + i] = G;
            }
        double psi, P[9], A[81];
        snh_density(F, mu, lam, &psi, P, A);
        const double wd = w * det;
        *E += wd * psi;
        if (g)
            for (int c = 0; c < n3; ++c) {
                double sg = 0.0;
                for (int r = 0; r < 9; ++r) sg += B[r * n3 + c] * P[r];
                g[c] += wd * sg;
            }
        if (H) {
            if (project) orc_clamp_psd(9, A);
            for (int r = 0; r < n3; ++r)
                for (int c = 0; c < n3; ++c) {
                    double sh = 0.0;
                    for (int k = 0; k < 9; ++k) {
                        if (B[k * n3 + r] == 0.0) continue;
                        double ab = 0.0;
                        for (int l = 0; l < 9; ++l) ab += A[k * 9 + l] * B[l * n3 + c];
                        sh += B[k * n3 + r] * ab;
                    }
                    H[(size_t)r * n3 + c] += wd * sh;
                }
        }
    }
    return bad;
}

/* A batch of T elements (tets: T x K node ids; X rest, x current: node
 * arrays). E_e (T), g_e (T x 3K), H_e (T x 3K x 3K). Returns the number of
 * elements with a non-positive det(J0) at some point. */
int orc_tetho_batch(int K, int T, const double* X, const double* x, const int* tets, int nq,
                    const double* rule, const double* mu, const double* lam, int level,
                    int project, double* E_e, double* g_e, double* H_e)
{
    int bad = 0, n3 = 3 * K;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
    for (int e = 0; e < T; ++e) {
        double Xe[60], xe[60];
        for (int a = 0; a < K; ++a)
            for (int i = 0; i < 3; ++i) {
                Xe[3 * a + i] = X[3 * (size_t)tets[K * (size_t)e + a] + i];
                xe[3 * a + i] = x[3 * (size_t)tets[K * (size_t)e + a] + i];
            }
        bad += orc_tetho_element(K, nq, rule, Xe, xe, mu[e], lam[e], project, E_e + e,
                                 level >= 1 ? g_e + (size_t)n3 * e : NULL,
                                 level >= 2 ? H_e + (size_t)n3 * n3 * e : NULL);
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* 3x3 block CRS pattern and slot maps (§5.3)                           */
/* ------------------------------------------------------------------ */

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* Pattern = union over all stencils of their node pairs, plus the
 * diagonal of every node; full storage, columns ascending in each row.
 * Call with col == NULL to get row_ptr and the block count, then again
 * with col sized to that count. READING: full (both triangles) storage,
 * int32 indices. */
long long orc_bsr_pattern(int N, int nst, const int* conn, int* row_ptr, int* col)
{
    int* cnt = (int*)calloc((size_t)N, sizeof(int));
    for (int e = 0; e < nst; ++e)
        for (int a = 0; a < 4; ++a) cnt[conn[4 * e + a]] += 4;
    size_t* off = (size_t*)malloc(((size_t)N + 1) * sizeof(size_t));
    off[0] = 0;
    for (int n = 0; n < N; ++n) off[n + 1] = off[n] + (size_t)cnt[n] + 1;
    int* buf = (int*)malloc(off[N] * sizeof(int));
    int* fill = (int*)calloc((size_t)N, sizeof(int));
    for (int n = 0; n < N; ++n) buf[off[n] + fill[n]++] = n;
    for (int e = 0; e < nst; ++e)
        for (int a = 0; a < 4; ++a) {
            int r = conn[4 * e + a];
            for (int b = 0; b < 4; ++b) buf[off[r] + fill[r]++] = conn[4 * e + b];
        }
    long long nnz = 0;
    row_ptr[0] = 0;
    for (int n = 0; n < N; ++n) {
        int* row = buf + off[n];
        int len = fill[n];
        qsort(row, (size_t)len, sizeof(int), cmp_int);
        int u = 0;
        for (int k = 0; k < len; ++k)
            if (k == 0 || row[k] != row[k - 1]) {
                if (col) col[nnz + u] = row[k];
                u++;
            }
        nnz += u;
        row_ptr[n + 1] = (int)nnz;
    }
    free(cnt); free(off); free(buf); free(fill);
    return nnz;
}

static int find_slot(const int* row_ptr, const int* col, int r, int c)
{
    int lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (col[mid] == c) return mid;
        if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* slots[16 e + 4 a + b] = block index of (node a, node b) of stencil e;
 * diag_slot[n] = block index of (n, n). */
void orc_bsr_slots(int N, const int* row_ptr, const int* col, int nst,
                   const int* conn, int* slots, int* diag_slot)
{
    for (int e = 0; e < nst; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                slots[16 * (size_t)e + 4 * a + b] =
                    find_slot(row_ptr, col, conn[4 * e + a], conn[4 * e + b]);
    for (int n = 0; n < N; ++n) diag_slot[n] = find_slot(row_ptr, col, n, n);
}

/* ------------------------------------------------------------------ */
/* Assembly (Algorithm 1; gradient sum R_e^T g_e)                       */
/* ------------------------------------------------------------------ */

/* Adds element blocks in stencil order (vals and grad must be zeroed by
 * the caller or hold earlier contributions). H_e may be NULL. */
void orc_assemble_elements(int nst, const int* conn, const int* slots,
                           const double* g_e, const double* H_e,
                           double* grad, double* vals)
{
    for (int e = 0; e < nst; ++e)
        for (int a = 0; a < 4; ++a) {
            int na = conn[4 * e + a];
            if (grad)
                for (int i = 0; i < 3; ++i) grad[3 * na + i] += g_e[12 * (size_t)e + 3 * a + i];
            if (H_e && vals)
                for (int b = 0; b < 4; ++b) {
                    double* blk = vals + 9 * (size_t)slots[16 * (size_t)e + 4 * a + b];
                    const double* He = H_e + 144 * (size_t)e;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j)
                            blk[3 * i + j] += He[(3 * a + i) * 12 + (3 * b + j)];
                }
        }
}

/* Inertia of the incremental potential (Eq. 2): per node
 * m/(2 dt^2) |x - xt|^2, gradient m/dt^2 (x - xt), diagonal m/dt^2 I.
 * With x0 != NULL, `xt` holds the increment xt - x0 (= dt v + dt^2 g) and
 * the residual is formed as (x - x0) - (xt - x0): the first difference is
 * exact for nearby x and x0, which keeps E_BE free of the O(|x| eps)
 * rounding that would otherwise swamp the last Newton decreases. */
static double inertia_impl(int N, const double* m, double dt, const double* x,
                           const double* x0, const double* xt, const int* diag_slot,
                           double* grad, double* vals)
{
    double E = 0.0, inv = 1.0 / (dt * dt);
    for (int n = 0; n < N; ++n) {
        double r2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            double r = x0 ? (x[3 * n + i] - x0[3 * n + i]) - xt[3 * n + i]
                          : x[3 * n + i] - xt[3 * n + i];
            r2 += r * r;
            if (grad) grad[3 * n + i] += m[n] * inv * r;
        }
        E += 0.5 * m[n] * inv * r2;
        if (vals && diag_slot)
            for (int i = 0; i < 3; ++i) vals[9 * (size_t)diag_slot[n] + 4 * i] += m[n] * inv;
    }
    return E;
}

double orc_inertia(int N, const double* m, double dt, const double* x,
                   const double* xt, const int* diag_slot, double* grad, double* vals)
{
    return inertia_impl(N, m, dt, x, NULL, xt, diag_slot, grad, vals);
}

/* ------------------------------------------------------------------ */
/* Block-Jacobi PCG (§7.2)                                              */
/* ------------------------------------------------------------------ */

/* y = A x with pinned rows/columns eliminated: pinned DOFs map to
 * themselves (identity), free rows only see free columns. READING: the
 * paper leaves Dirichlet handling open; DOF elimination by mask is used. */
static void spmv_masked(int N, const int* rp, const int* col, const double* vals,
                        const unsigned char* pinned, const double* x, double* y)
{
    for (int r = 0; r < N; ++r) {
        if (pinned && pinned[r]) {
            for (int i = 0; i < 3; ++i) y[3 * r + i] = x[3 * r + i];
            continue;
        }
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = rp[r]; k < rp[r + 1]; ++k) {
            int c = col[k];
            if (pinned && pinned[c]) continue;
            const double* B = vals + 9 * (size_t)k;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc[i] += B[3 * i + j] * x[3 * c + j];
        }
        for (int i = 0; i < 3; ++i) y[3 * r + i] = acc[i];
    }
}

static double dotv(size_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Preconditioned CG on the masked system, x0 = 0, stop when
 * ||r||_2 <= tol ||b||_2. READING: a fixed tolerance instead of the
 * paper's forcing sequence. Returns 0, or ORC_ENOTCONV after maxit. */
int orc_pcg(int N, const int* rp, const int* col, const double* vals,
            const int* diag_slot, const unsigned char* pinned, const double* b,
            double tol, int maxit, double* x, int* iters, double* relres)
{
    size_t n3 = 3 * (size_t)N;
    double* Minv = (double*)malloc(9 * (size_t)N * sizeof(double));
    double *r = (double*)malloc(n3 * sizeof(double)), *z = (double*)malloc(n3 * sizeof(double));
    double *p = (double*)malloc(n3 * sizeof(double)), *q = (double*)malloc(n3 * sizeof(double));
    for (int n = 0; n < N; ++n) {
        if (pinned && pinned[n]) {
            for (int k = 0; k < 9; ++k) Minv[9 * n + k] = (k % 4 == 0) ? 1.0 : 0.0;
        } else {
            inv3(vals + 9 * (size_t)diag_slot[n], Minv + 9 * (size_t)n, NULL);
        }
    }
    for (size_t i = 0; i < n3; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bn = sqrt(dotv(n3, b, b));
    int it = 0, status = 0;
    double rn = bn;
    if (bn == 0.0) goto done;
#define APPLY_M(dst, src) \
    for (int nn = 0; nn < N; ++nn) \
        for (int i = 0; i < 3; ++i) { \
            double s_ = 0.0; \
            for (int j = 0; j < 3; ++j) s_ += Minv[9 * (size_t)nn + 3 * i + j] * (src)[3 * nn + j]; \
            (dst)[3 * nn + i] = s_; \
        }
    APPLY_M(z, r);
    for (size_t i = 0; i < n3; ++i) p[i] = z[i];
    double rz = dotv(n3, r, z);
    status = ORC_ENOTCONV;
    for (it = 0; it < maxit;) {
        spmv_masked(N, rp, col, vals, pinned, p, q);
        double alpha = rz / dotv(n3, p, q);
        for (size_t i = 0; i < n3; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        rn = sqrt(dotv(n3, r, r));
        if (rn <= tol * bn) { status = 0; break; }
        APPLY_M(z, r);
        double rz2 = dotv(n3, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (size_t i = 0; i < n3; ++i) p[i] = z[i] + beta * p[i];
    }
#undef APPLY_M
done:
    if (iters) *iters = it;
    if (relres) *relres = (bn > 0.0) ? rn / bn : 0.0;
    free(Minv); free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* Scene evaluation and the backward-Euler Newton step (Eqs. 2-3)       */
/* ------------------------------------------------------------------ */

typedef struct {
    int N;
    const double* mass;
    int n_snh;
    const int* snh_tets;
    const double* snh_Dminv;
    const double* snh_V;
    const double* snh_mu;
    const double* snh_lam;
    int n_hinge;
    const int* hinge;
    const double* hinge_q;
    const double* hinge_c;
    double kb;
    int n_pt;
    const int* pt;
    double dhat;
    double kappa;
    const unsigned char* pinned;
    /* pattern over the concatenated stencils (snh, hinge, pt) */
    const int* row_ptr;
    const int* col;
    const int* slots;
    const int* diag_slot;
    long long nnzb;
    /* density of the tet block (ORC_MODEL_*) and its lagged rotations
     * (9 per tet, COROT / ARAP) */
    int snh_model;
    const double* snh_R;
    /* lagged friction block on point-triangle pairs: its lag data is taken
     * at the start of every Newton step (orc_newton_step writes it) */
    int n_fr;
    const int* fr;
    double fr_mu, fr_yhat, fr_dhat, fr_kappa;
    double* fr_beta;
    double* fr_T;
    double* fr_fn;
    double* fr_dxt;
} orc_scene;

/* Full evaluation of E_BE = inertia + sum of element energies at x
 * (Eq. 2 with Eq. 5). level as above. Returns the number of stencils in
 * an invalid state (barrier d <= 0, Neo-Hookean J <= 0). grad/vals are
 * overwritten. */
static int scene_eval_impl(const orc_scene* s, const double* x, const double* x0,
                           const double* xt, double dt, int level, int project,
                           double* E_out, double* grad, double* vals)
{
    int bad = 0;
    size_t n3 = 3 * (size_t)s->N;
    if (level >= 1) memset(grad, 0, n3 * sizeof(double));
    if (level >= 2) memset(vals, 0, 9 * (size_t)s->nnzb * sizeof(double));
    double E = 0.0;
    size_t base = 0;
    int counts[4] = {s->n_snh, s->n_hinge, s->n_pt, s->n_fr};
    for (int kind = 0; kind < 4; ++kind) {
        int n = counts[kind];
        if (n == 0) continue;
        double* Ee = (double*)malloc((size_t)n * sizeof(double));
        double* ge = level >= 1 ? (double*)malloc(12 * (size_t)n * sizeof(double)) : NULL;
        double* He = level >= 2 ? (double*)malloc(144 * (size_t)n * sizeof(double)) : NULL;
        const int* conn;
        if (kind == 0) {
            conn = s->snh_tets;
            bad += orc_tet_batch(s->snh_model, n, x, conn, s->snh_Dminv, s->snh_V, s->snh_mu,
                                 s->snh_lam, s->snh_R, level, project, Ee, ge, He);
        } else if (kind == 1) {
            conn = s->hinge;
            orc_hinge_batch(n, x, conn, s->hinge_q, s->hinge_c, s->kb, level, Ee, ge, He);
        } else if (kind == 2) {
            conn = s->pt;
            bad += orc_barrier_batch(n, x, conn, s->dhat, s->kappa, level, project,
                                     Ee, ge, He, NULL);
        } else {
            /* friction: PSD by construction, never projected */
            conn = s->fr;
            orc_friction_batch(n, x, conn, s->fr_beta, s->fr_T, s->fr_fn, s->fr_dxt, s->fr_mu,
                               s->fr_yhat, dt, level, Ee, ge, He);
        }
        for (int e = 0; e < n; ++e) E += Ee[e];
        if (level >= 1)
            orc_assemble_elements(n, conn, s->slots + 16 * base, ge, He, grad,
                                  level >= 2 ? vals : NULL);
        free(Ee); free(ge); free(He);
        base += (size_t)n;
    }
    if (xt && s->mass)
        E += inertia_impl(s->N, s->mass, dt, x, x0, xt, s->diag_slot,
                          level >= 1 ? grad : NULL, level >= 2 ? vals : NULL);
    *E_out = E;
    return bad;
}

int orc_scene_eval(const orc_scene* s, const double* x, const double* xt, double dt,
                   int level, int project, double* E_out, double* grad, double* vals)
{
    return scene_eval_impl(s, x, NULL, xt, dt, level, project, E_out, grad, vals);
}

typedef struct {
    double newton_tol;
    double pcg_tol;
    int max_newton;
    int max_pcg;
    int max_halvings;
    double armijo_c;
    int project;
    /* 1: the PCG tolerance of Newton iteration k is the forcing term
     * max(pcg_tol, min(1/2, sqrt(||g_k|| / ||g_0||))) (READING of the §7.2
     * solver paragraph, which names a forcing sequence without a formula) */
    int forcing;
} orc_newton_opts;

typedef struct {
    int status;
    int newton_iters;
    int pcg_iters_total;
    double g0_norm;
    double g_norm;
    double E_final;
} orc_newton_report;

static double free_norm(int N, const unsigned char* pinned, const double* g)
{
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
        if (pinned && pinned[n]) continue;
        for (int i = 0; i < 3; ++i) s += g[3 * n + i] * g[3 * n + i];
    }
    return sqrt(s);
}

/* One backward-Euler step (Eqs. 2-3): xt = x + dt v + dt^2 g_ext;
 * Newton from x0 = x_t (READING) with PCG directions and backtracking
 * Armijo line search; stop when ||g_free|| <= tol max(||g_free(x0)||,
 * ||M g_ext||_free, 1e-30) (READING); then v = (x - x_t)/dt. x and v are
 * updated in place. */
int orc_newton_step(const orc_scene* s, double dt, const double gravity[3],
                    const orc_newton_opts* o, double* x, double* v,
                    orc_newton_report* rep)
{
    int N = s->N;
    size_t n3 = 3 * (size_t)N;
    double *xt = (double*)malloc(n3 * sizeof(double)), *x0 = (double*)malloc(n3 * sizeof(double));
    double *g = (double*)malloc(n3 * sizeof(double)), *gtr = (double*)malloc(n3 * sizeof(double));
    double *dx = (double*)malloc(n3 * sizeof(double)), *b = (double*)malloc(n3 * sizeof(double));
    double *xtr = (double*)malloc(n3 * sizeof(double));
    double* vals = (double*)malloc(9 * (size_t)s->nnzb * sizeof(double));
    for (int n = 0; n < N; ++n)
        for (int i = 0; i < 3; ++i) {
            x0[3 * n + i] = x[3 * n + i];
            /* increment xt - x0 = dt v + dt^2 g (Eq. 2) */
            xt[3 * n + i] = dt * v[3 * n + i] + dt * dt * gravity[i];
        }
    /* lagged friction data at the start-of-step state */
    if (s->n_fr)
        orc_friction_lag_batch(s->n_fr, x0, s->fr, s->fr_dhat, s->fr_kappa, s->fr_beta, s->fr_T,
                               s->fr_fn, s->fr_dxt);
    int status = ORC_ENOTCONV, it = 0, pcg_total = 0;
    double E, gn0 = 0.0, gn = 0.0;
    double fext = 0.0;   /* || M g_ext || over the free DOFs */
    if (s->mass) {
        double g2 = gravity[0] * gravity[0] + gravity[1] * gravity[1] + gravity[2] * gravity[2];
        for (int n = 0; n < N; ++n)
            if (!(s->pinned && s->pinned[n])) fext += s->mass[n] * s->mass[n] * g2;
        fext = sqrt(fext);
    }
    for (it = 0; it <= o->max_newton; ++it) {
        scene_eval_impl(s, x, x0, xt, dt, 2, o->project, &E, g, vals);
        gn = free_norm(N, s->pinned, g);
        if (it == 0) gn0 = gn;
        /* READING: the residual is measured against the larger of the
         * initial residual and the external force on the free DOFs, so a
         * scene that starts the step near equilibrium is not asked for a
         * residual below the rounding of its own gradient */
        double ref = gn0 > fext ? gn0 : fext;
        if (ref < 1e-30) ref = 1e-30;
        if (gn <= o->newton_tol * ref) { status = 0; break; }
        if (it == o->max_newton) break;
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < 3; ++i)
                b[3 * n + i] = (s->pinned && s->pinned[n]) ? 0.0 : -g[3 * n + i];
        double ptol = o->pcg_tol;
        if (o->forcing) {
            double eta = sqrt(gn / (gn0 > 1e-300 ? gn0 : 1e-300));
            if (eta > 0.5) eta = 0.5;
            if (eta > ptol) ptol = eta;
        }
        int pit = 0;
        int pst = orc_pcg(N, s->row_ptr, s->col, vals, s->diag_slot, s->pinned, b,
                          ptol, o->max_pcg, dx, &pit, NULL);
        pcg_total += pit;
        if (pst != 0) { status = ORC_ENOTCONV; break; }
        double gdx = dotv(n3, g, dx);
        double alpha = 1.0;
        int accepted = 0;
        for (int h = 0; h <= o->max_halvings; ++h) {
            for (size_t k = 0; k < n3; ++k) xtr[k] = x[k] + alpha * dx[k];
            double Et;
            int bad = scene_eval_impl(s, xtr, x0, xt, dt, 0, 0, &Et, NULL, NULL);
            /* READING: once the predicted decrease is below what double
             * energies resolve (|g.dx| < 1e-12 |E|), the energy comparison
             * carries no information and the full Newton step is taken */
            int tiny = fabs(gdx) < 1e-12 * fabs(E);
            if (bad == 0 && isfinite(Et) && (tiny || Et <= E + o->armijo_c * alpha * gdx)) {
                accepted = 1;
                break;
            }
            alpha *= 0.5;
        }
        if (!accepted) { status = ORC_ELINESEARCH; break; }
        memcpy(x, xtr, n3 * sizeof(double));
    }
    for (size_t k = 0; k < n3; ++k) v[k] = (x[k] - x0[k]) / dt;
    if (rep) {
        rep->status = status;
        rep->newton_iters = it;
        rep->pcg_iters_total = pcg_total;
        rep->g0_norm = gn0;
        rep->g_norm = gn;
        rep->E_final = E;
    }
    free(xt); free(x0); free(g); free(gtr); free(dx); free(b); free(xtr); free(vals);
    return status;
}
