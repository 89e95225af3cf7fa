/*
 * Nekbone oracle: a plain, slow, obviously correct FP64 CPU restatement of
 * the spectral-element Poisson hot path studied in Karp et al.,
 * "Optimization of Tensor-product Operations in Nekbone on GPUs"
 * (arXiv 2005.13425).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the
 * CUDA library.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA path, and the CUDA path never calls it.
 *
 * Everything is IEEE double, compiled without FMA contraction
 * (-ffp-contract=off) so each expression rounds exactly as written.
 * Loops are in the order of the definitions they restate; the only
 * concurrency is an optional OpenMP loop over elements in nbo_ax_e, whose
 * elements are independent, so its result does not depend on the thread
 * count.
 *
 * Notation (paper Sec. III and III.A):
 *   n      GLL points per direction, n = degree + 1, N = n - 1 the degree
 *   E      number of elements (nelt), a box of Ex x Ey x Ez hexahedra,
 *          element id e = ex + Ex*(ey + Ey*ez)
 *   local storage  u[e][k][j][i], i fastest: u[e*n^3 + i + n*(j + n*k)]
 *   D      dxm1, row major D[i*n + l] = dxm1(i,l) = l_l'(xi_i)
 *   gxyz   [E][6][n^3], components rr, rs, rt, ss, st, tt (Listing 1's 1..6)
 *
 * Pins: every function here is checked by the `-m "not gpu"` tests against
 * closed forms, invariants, brute force or library routines (GLL quadrature
 * exactness, D applied to polynomials, A*1 = 0, symmetry, positivity, a
 * brute-force element matrix from an independent Lagrange-basis formula,
 * exact stiffness on affine elements, the isoparametric identity
 * x_c^T A x_a = delta_ca * sum(w detJ), coordinate-based numbering, a dense
 * library solve of the assembled system and a manufactured solution).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NBO_PI 3.14159265358979323846264338327950288L

/* ------------------------------------------------------------------ */
/* C1. Gauss-Lobatto-Legendre nodes and weights (textbook definition:  */
/* xi_0 = -1, xi_N = 1, interior nodes the roots of P_N'; weights      */
/* w_i = 2 / (N (N+1) P_N(xi_i)^2)).  Paper Sec. III.A names the GLL    */
/* points; the formulas are those of Canuto et al. / Deville et al.    */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_N and its derivative at x by the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and
 * P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void nbo_legendre(int N, long double x, long double *pN, long double *dpN)
{
    long double p0 = 1.0L, p1 = x;        /* P_0, P_1 */
    long double d0 = 0.0L, d1 = 1.0L;     /* P_0', P_1' */
    if (N == 0) { *pN = 1.0L; *dpN = 0.0L; return; }
    for (int k = 1; k < N; k++) {
        long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        long double d2 = d0 + (2 * k + 1) * p1;
        p0 = p1; p1 = p2;
        d0 = d1; d1 = d2;
    }
    *pN = p1;
    *dpN = d1;
}

/* Returns 0 on success, -1 on bad n. xi and w have n entries. */
int nbo_gll(int n, double *xi, double *w)
{
    if (n < 2) return -1;
    const int N = n - 1;
    for (int i = 0; i < n; i++) {
        long double x;
        if (i == 0) {
            x = -1.0L;
        } else if (i == N) {
            x = 1.0L;
        } else {
            /* Newton on q(x) = P_N'(x) from the Chebyshev-Gauss-Lobatto guess.
             * q'(x) = P_N''(x) = (2x P_N' - N(N+1) P_N) / (1 - x^2)
             * from Legendre's equation. */
            x = -cosl(NBO_PI * (long double)i / (long double)N);
            for (int it = 0; it < 100; it++) {
                long double p, dp;
                nbo_legendre(N, x, &p, &dp);
                long double d2p = (2.0L * x * dp - (long double)N * (N + 1) * p) / (1.0L - x * x);
                long double dx = dp / d2p;
                x -= dx;
                if (fabsl(dx) < 1e-30L) break;
            }
        }
        long double p, dp;
        nbo_legendre(N, x, &p, &dp);
        xi[i] = (double)x;
        w[i] = (double)(2.0L / ((long double)N * (N + 1) * p * p));
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* C2. Derivative matrix dxm1(i,l) = l_l'(xi_i) (Listing 1's dxm1):    */
/*   i != l : P_N(xi_i) / (P_N(xi_l) (xi_i - xi_l))                    */
/*   (0,0)  : -N(N+1)/4,  (N,N) : N(N+1)/4,  other diagonal entries 0. */
/* Stored row major, D[i*n + l].  dxtm1 = D^T.                          */
/* ------------------------------------------------------------------ */
int nbo_dmat(int n, const double *xi, double *D)
{
    if (n < 2) return -1;
    const int N = n - 1;
    for (int i = 0; i < n; i++) {
        for (int l = 0; l < n; l++) {
            long double v;
            if (i != l) {
                long double pi, dpi, pl, dpl;
                nbo_legendre(N, (long double)xi[i], &pi, &dpi);
                nbo_legendre(N, (long double)xi[l], &pl, &dpl);
                v = pi / (pl * ((long double)xi[i] - (long double)xi[l]));
            } else if (i == 0) {
                v = -(long double)N * (N + 1) / 4.0L;
            } else if (i == N) {
                v = (long double)N * (N + 1) / 4.0L;
            } else {
                v = 0.0L;
            }
            D[i * n + l] = (double)v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* C3. Box mesh and geometric factors.                                 */
/* Unit cube split into Ex x Ey x Ez elements; element (ex,ey,ez) maps  */
/* the reference cube [-1,1]^3 to [ex/Ex,(ex+1)/Ex] x ... (affine box   */
/* X), then the smooth perturbation                                     */
/*   x_d = X_d + amp * s_d * sin(pi X) sin(pi Y) sin(pi Z),  d = 1..3, */
/* which vanishes on the boundary of the cube.                          */
/* ------------------------------------------------------------------ */

/* Nodal physical coordinates, xyz[e][d][n^3] with d = x, y, z. */
int nbo_box_coords(int Ex, int Ey, int Ez, int n, const double *xi,
                   double amp, const double *s, double *xyz)
{
    if (Ex < 1 || Ey < 1 || Ez < 1 || n < 2) return -1;
    const long n3 = (long)n * n * n;
    for (int ez = 0; ez < Ez; ez++)
    for (int ey = 0; ey < Ey; ey++)
    for (int ex = 0; ex < Ex; ex++) {
        long e = ex + (long)Ex * (ey + (long)Ey * ez);
        for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            double X = (ex + 0.5 * (xi[i] + 1.0)) / Ex;
            double Y = (ey + 0.5 * (xi[j] + 1.0)) / Ey;
            double Z = (ez + 0.5 * (xi[k] + 1.0)) / Ez;
            double bump = sin(M_PI * X) * sin(M_PI * Y) * sin(M_PI * Z);
            long p = i + n * (j + (long)n * k);
            xyz[e * 3 * n3 + 0 * n3 + p] = X + amp * s[0] * bump;
            xyz[e * 3 * n3 + 1 * n3 + p] = Y + amp * s[1] * bump;
            xyz[e * 3 * n3 + 2 * n3 + p] = Z + amp * s[2] * bump;
        }
    }
    return 0;
}

/* Geometric factors gxyz = w_i w_j w_k |J| J^{-1} J^{-T}, with the
 * Jacobian J_ab = dx_a/dr_b obtained isoparametrically by applying D to
 * the nodal coordinates along r (index i), s (j) and t (k).
 * G_bc = sum_m (dr_b/dx_m)(dr_c/dx_m).  Component order rr, rs, rt, ss,
 * st, tt, as Listing 1 uses gxyz(.,1..6).  detJ (optional) receives |J|
 * per point.  Returns -2 if some |J| <= 0. */
int nbo_geom(int E, int n, const double *D, const double *wgll,
             const double *xyz, double *gxyz, double *detJ)
{
    const long n3 = (long)n * n * n;
    int bad = 0;
    for (long e = 0; e < E; e++) {
        for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            long p = i + n * (j + (long)n * k);
            double J[3][3];
            for (int a = 0; a < 3; a++) {
                const double *x = xyz + e * 3 * n3 + a * n3;
                double dr = 0.0, ds = 0.0, dt = 0.0;
                for (int l = 0; l < n; l++) {
                    dr = dr + D[i * n + l] * x[l + n * (j + (long)n * k)];
                    ds = ds + D[j * n + l] * x[i + n * (l + (long)n * k)];
                    dt = dt + D[k * n + l] * x[i + n * (j + (long)n * l)];
                }
                J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
            }
            double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                       - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                       + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            if (!(det > 0.0)) bad = 1;
            /* Inverse by the adjugate: Jinv[b][m] = dr_b/dx_m. */
            double Jinv[3][3];
            Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
            Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
            Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
            Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
            Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
            Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
            Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
            Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
            Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
            double G[3][3];
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    double g = 0.0;
                    for (int m = 0; m < 3; m++) g = g + Jinv[b][m] * Jinv[c][m];
                    G[b][c] = g;
                }
            double scale = wgll[i] * wgll[j] * wgll[k] * det;
            double *g6 = gxyz + e * 6 * n3;
            g6[0 * n3 + p] = scale * G[0][0];
            g6[1 * n3 + p] = scale * G[0][1];
            g6[2 * n3 + p] = scale * G[0][2];
            g6[3 * n3 + p] = scale * G[1][1];
            g6[4 * n3 + p] = scale * G[1][2];
            g6[5 * n3 + p] = scale * G[2][2];
            if (detJ) detJ[e * n3 + p] = det;
        }
    }
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* C4. ax_e, Listing 1 restated loop for loop.                         */
/* First loop nest: wr, ws, wt = dxm1 applied along r, s, t, then       */
/* ur, us, ut = the symmetric 3x3 gxyz contraction.  Second loop nest:  */
/* w = sum_l dxtm1(i,l) ur(l,j,k) + dxtm1(j,l) us(i,l,k)                */
/*               + dxtm1(k,l) ut(i,j,l),   dxtm1(i,l) = dxm1(l,i).      */
/* ------------------------------------------------------------------ */
void nbo_ax_e(int E, int n, const double *D, const double *gxyz,
              const double *u, double *w)
{
    const long n3 = (long)n * n * n;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double *ur = (double *)malloc(sizeof(double) * 3 * n3);
        double *us = ur + n3;
        double *ut = us + n3;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long e = 0; e < E; e++) {
            const double *ue = u + e * n3;
            const double *g = gxyz + e * 6 * n3;
            double *we = w + e * n3;
            for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double wr = 0.0, ws = 0.0, wt = 0.0;
                for (int l = 0; l < n; l++) {
                    wr = wr + D[i * n + l] * ue[l + n * (j + (long)n * k)];
                    ws = ws + D[j * n + l] * ue[i + n * (l + (long)n * k)];
                    wt = wt + D[k * n + l] * ue[i + n * (j + (long)n * l)];
                }
                long p = i + n * (j + (long)n * k);
                ur[p] = g[0 * n3 + p] * wr + g[1 * n3 + p] * ws + g[2 * n3 + p] * wt;
                us[p] = g[1 * n3 + p] * wr + g[3 * n3 + p] * ws + g[4 * n3 + p] * wt;
                ut[p] = g[2 * n3 + p] * wr + g[4 * n3 + p] * ws + g[5 * n3 + p] * wt;
            }
            for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                long p = i + n * (j + (long)n * k);
                double acc = 0.0;
                for (int l = 0; l < n; l++) {
                    /* dxtm1(i,l) = dxm1(l,i) = D[l*n + i] */
                    acc = acc + D[l * n + i] * ur[l + n * (j + (long)n * k)]
                              + D[l * n + j] * us[i + n * (l + (long)n * k)]
                              + D[l * n + k] * ut[i + n * (j + (long)n * l)];
                }
                we[p] = acc;
            }
        }
        free(ur);
    }
}

/* ------------------------------------------------------------------ */
/* C5. Direct stiffness summation and mask on the box mesh.            */
/* Global node of local point (e; i,j,k):                               */
/*   (gx, gy, gz) = (ex (n-1) + i, ey (n-1) + j, ez (n-1) + k)          */
/*   gid = gx + NX (gy + NY gz),  NX = Ex (n-1) + 1, NY, NZ likewise.   */
/* ------------------------------------------------------------------ */
void nbo_gid(int Ex, int Ey, int Ez, int n, int64_t *gid)
{
    const long n3 = (long)n * n * n;
    const long NX = (long)Ex * (n - 1) + 1, NY = (long)Ey * (n - 1) + 1;
    for (int ez = 0; ez < Ez; ez++)
    for (int ey = 0; ey < Ey; ey++)
    for (int ex = 0; ex < Ex; ex++) {
        long e = ex + (long)Ex * (ey + (long)Ey * ez);
        for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            long gx = (long)ex * (n - 1) + i;
            long gy = (long)ey * (n - 1) + j;
            long gz = (long)ez * (n - 1) + k;
            gid[e * n3 + i + n * (j + (long)n * k)] = gx + NX * (gy + NY * gz);
        }
    }
}

/* Number of local copies of each local point's global node. */
void nbo_multiplicity(int Ex, int Ey, int Ez, int n, int32_t *mult)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n;
    const long NX = (long)Ex * (n - 1) + 1, NY = (long)Ey * (n - 1) + 1,
               NZ = (long)Ez * (n - 1) + 1;
    int64_t *gid = (int64_t *)malloc(sizeof(int64_t) * E * n3);
    int32_t *count = (int32_t *)calloc(NX * NY * NZ, sizeof(int32_t));
    nbo_gid(Ex, Ey, Ez, n, gid);
    for (long q = 0; q < E * n3; q++) count[gid[q]] += 1;
    for (long q = 0; q < E * n3; q++) mult[q] = count[gid[q]];
    free(count);
    free(gid);
}

/* Homogeneous Dirichlet mask on all six faces of the box:
 * mask = 0 where the global node lies on the boundary, else 1. */
void nbo_mask(int Ex, int Ey, int Ez, int n, uint8_t *mask)
{
    const long n3 = (long)n * n * n;
    const long NX = (long)Ex * (n - 1) + 1, NY = (long)Ey * (n - 1) + 1,
               NZ = (long)Ez * (n - 1) + 1;
    for (int ez = 0; ez < Ez; ez++)
    for (int ey = 0; ey < Ey; ey++)
    for (int ex = 0; ex < Ex; ex++) {
        long e = ex + (long)Ex * (ey + (long)Ey * ez);
        for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            long gx = (long)ex * (n - 1) + i;
            long gy = (long)ey * (n - 1) + j;
            long gz = (long)ez * (n - 1) + k;
            int on_bdry = gx == 0 || gx == NX - 1 || gy == 0 || gy == NY - 1 ||
                          gz == 0 || gz == NZ - 1;
            mask[e * n3 + i + n * (j + (long)n * k)] = on_bdry ? 0 : 1;
        }
    }
}

/* dssum: every global node's value becomes the sum of its local copies,
 * accumulated from +0.0 in ascending (element id, local index) order,
 * and that sum is written back to every copy. */
void nbo_dssum(int Ex, int Ey, int Ez, int n, double *w)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n;
    const long NX = (long)Ex * (n - 1) + 1, NY = (long)Ey * (n - 1) + 1,
               NZ = (long)Ez * (n - 1) + 1;
    int64_t *gid = (int64_t *)malloc(sizeof(int64_t) * E * n3);
    double *acc = (double *)malloc(sizeof(double) * NX * NY * NZ);
    nbo_gid(Ex, Ey, Ez, n, gid);
    for (long g = 0; g < NX * NY * NZ; g++) acc[g] = 0.0;
    for (long q = 0; q < E * n3; q++) acc[gid[q]] = acc[gid[q]] + w[q];
    for (long q = 0; q < E * n3; q++) w[q] = acc[gid[q]];
    free(acc);
    free(gid);
}

/* Mask: w := +0.0 where mask == 0 (a select, not a product). */
void nbo_apply_mask(long npts, const uint8_t *mask, double *w)
{
    for (long q = 0; q < npts; q++)
        if (mask[q] == 0) w[q] = 0.0;
}

/* Weighted inner product <a,b>_c = sum_local a b c, c = 1/multiplicity,
 * summed sequentially over elements, then local index.  Equals the dot
 * product over unique nodes for vectors that are continuous. */
double nbo_dot_c(int Ex, int Ey, int Ez, int n, const double *a, const double *b)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n;
    int32_t *mult = (int32_t *)malloc(sizeof(int32_t) * E * n3);
    nbo_multiplicity(Ex, Ey, Ez, n, mult);
    double s = 0.0;
    for (long q = 0; q < E * n3; q++) s = s + a[q] * b[q] * (1.0 / mult[q]);
    free(mult);
    return s;
}

/* The assembled operator A u = mask(dssum(ax_e(u))). */
void nbo_apply_A(int Ex, int Ey, int Ez, int n, const double *D, const double *gxyz,
                 const uint8_t *mask, const double *u, double *w)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n;
    nbo_ax_e((int)E, n, D, gxyz, u, w);
    nbo_dssum(Ex, Ey, Ez, n, w);
    nbo_apply_mask(E * n3, mask, w);
}

/* ------------------------------------------------------------------ */
/* Jacobi preconditioner (the paper names preconditioned CG as future   */
/* work, Sec. VII).  The diagonal of the element matrix A_e of Listing 1 */
/* at local point p = (i,j,k) is sum over quadrature points of          */
/* grad(phi_p)^T G grad(phi_p); d/dr phi_p is nonzero only on the line  */
/* through p along r (value dxm1(a,i) at node a), and likewise for s, t, */
/* so                                                                   */
/*   A_e(p,p) = sum_a D(a,i)^2 g_rr(a,j,k) + sum_b D(b,j)^2 g_ss(i,b,k) */
/*            + sum_c D(c,k)^2 g_tt(i,j,c)                               */
/*            + 2 D(i,i) D(j,j) g_rs(p) + 2 D(i,i) D(k,k) g_rt(p)        */
/*            + 2 D(j,j) D(k,k) g_st(p).                                 */
/* ------------------------------------------------------------------ */
void nbo_diag_e(int E, int n, const double *D, const double *gxyz, double *diag)
{
    const long n3 = (long)n * n * n;
    for (long e = 0; e < E; e++) {
        const double *g = gxyz + e * 6 * n3;
        for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            long p = i + n * (j + (long)n * k);
            double d = 0.0;
            for (int a = 0; a < n; a++)
                d = d + D[a * n + i] * D[a * n + i] * g[0 * n3 + a + n * (j + (long)n * k)];
            for (int b = 0; b < n; b++)
                d = d + D[b * n + j] * D[b * n + j] * g[3 * n3 + i + n * (b + (long)n * k)];
            for (int c = 0; c < n; c++)
                d = d + D[c * n + k] * D[c * n + k] * g[5 * n3 + i + n * (j + (long)n * c)];
            d = d + 2.0 * D[i * n + i] * D[j * n + j] * g[1 * n3 + p]
                  + 2.0 * D[i * n + i] * D[k * n + k] * g[2 * n3 + p]
                  + 2.0 * D[j * n + j] * D[k * n + k] * g[4 * n3 + p];
            diag[e * n3 + p] = d;
        }
    }
}

/* Inverse assembled diagonal: minv = 1 / dssum(diag_e) at unmasked points,
 * 0 at Dirichlet points. */
void nbo_jacobi_inverse(int Ex, int Ey, int Ez, int n, const double *D, const double *gxyz,
                        const uint8_t *mask, double *minv)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n;
    nbo_diag_e((int)E, n, D, gxyz, minv);
    nbo_dssum(Ex, Ey, Ez, n, minv);
    for (long q = 0; q < E * n3; q++) minv[q] = mask[q] ? 1.0 / minv[q] : 0.0;
}

/* ------------------------------------------------------------------ */
/* C6. Unpreconditioned conjugate gradient on local storage (Nekbone   */
/* form; the paper solves Ax = f with CG, Sec. III, and uses no         */
/* preconditioner, Sec. VII).                                            */
/*   r = f - A x0, rho_old = 1, p = 0                                   */
/*   for it = 1..maxit:                                                  */
/*     rho = <r,r>_c;  stop if tol > 0 and sqrt(rho)/sqrt(<f,f>_c) <= tol */
/*     beta = (it == 1) ? 0 : rho / rho_old;  p = r + beta p             */
/*     w = A p;  alpha = rho / <w,p>_c                                   */
/*     x = x + alpha p;  r = r - alpha w;  rho_old = rho                 */
/* tol <= 0 runs exactly maxit iterations.  rho_hist (optional) gets     */
/* rho_0 .. rho_iters (iters + 1 values), the last one after the final  */
/* update.  Returns 0, or 1 on breakdown (<w,p>_c <= 0 or not finite).  */
/* ------------------------------------------------------------------ */
int nbo_cg(int Ex, int Ey, int Ez, int n, const double *D, const double *gxyz,
           const uint8_t *mask, const double *f, double *x, double tol, int maxit,
           int *iters_out, double *relres_out, double *rho_hist)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n, npts = E * n3;
    double *r = (double *)malloc(sizeof(double) * npts);
    double *p = (double *)malloc(sizeof(double) * npts);
    double *w = (double *)malloc(sizeof(double) * npts);
    int status = 0, iters = 0;

    nbo_apply_A(Ex, Ey, Ez, n, D, gxyz, mask, x, w);
    for (long q = 0; q < npts; q++) { r[q] = f[q] - w[q]; p[q] = 0.0; }
    double fnorm = sqrt(nbo_dot_c(Ex, Ey, Ez, n, f, f));
    double rho_old = 1.0;
    double rho = nbo_dot_c(Ex, Ey, Ez, n, r, r);
    if (rho_hist) rho_hist[0] = rho;
    for (int it = 1; it <= maxit; it++) {
        if (rho == 0.0) break;
        if (tol > 0.0 && sqrt(rho) / fnorm <= tol) break;
        double beta = (it == 1) ? 0.0 : rho / rho_old;
        for (long q = 0; q < npts; q++) p[q] = r[q] + beta * p[q];
        nbo_apply_A(Ex, Ey, Ez, n, D, gxyz, mask, p, w);
        double pap = nbo_dot_c(Ex, Ey, Ez, n, w, p);
        if (!(pap > 0.0) || !isfinite(pap)) { status = 1; break; }
        double alpha = rho / pap;
        for (long q = 0; q < npts; q++) {
            x[q] = x[q] + alpha * p[q];
            r[q] = r[q] - alpha * w[q];
        }
        rho_old = rho;
        rho = nbo_dot_c(Ex, Ey, Ez, n, r, r);
        iters = it;
        if (rho_hist) rho_hist[it] = rho;
    }
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = fnorm > 0.0 ? sqrt(rho) / fnorm : 0.0;
    free(r); free(p); free(w);
    return status;
}

/* ------------------------------------------------------------------ */
/* Jacobi-preconditioned CG (textbook PCG, e.g. Saad, Iterative Methods */
/* for Sparse Linear Systems, Alg. 9.1) with z = minv .* r:             */
/*   r = f - A x0, z = minv r, p = 0, rho_old = 1                       */
/*   for it = 1..maxit:                                                  */
/*     rho = <r,z>_c; stop if rho == 0 or (tol > 0 and                   */
/*     sqrt(<r,r>_c / <f,f>_c) <= tol)                                   */
/*     beta = (it == 1) ? 0 : rho / rho_old;  p = z + beta p             */
/*     w = A p;  alpha = rho / <w,p>_c;  x += alpha p;  r -= alpha w     */
/*     z = minv r;  rho_old = rho                                         */
/* With minv = 1 this is nbo_cg step for step.  rr_hist (optional) gets */
/* <r,r>_c per iteration (iters + 1 values).                             */
/* ------------------------------------------------------------------ */
int nbo_pcg(int Ex, int Ey, int Ez, int n, const double *D, const double *gxyz,
            const uint8_t *mask, const double *minv, const double *f, double *x, double tol,
            int maxit, int *iters_out, double *relres_out, double *rr_hist)
{
    const long E = (long)Ex * Ey * Ez, n3 = (long)n * n * n, npts = E * n3;
    double *r = (double *)malloc(sizeof(double) * npts);
    double *z = (double *)malloc(sizeof(double) * npts);
    double *p = (double *)malloc(sizeof(double) * npts);
    double *w = (double *)malloc(sizeof(double) * npts);
    int status = 0, iters = 0;

    nbo_apply_A(Ex, Ey, Ez, n, D, gxyz, mask, x, w);
    for (long q = 0; q < npts; q++) { r[q] = f[q] - w[q]; z[q] = minv[q] * r[q]; p[q] = 0.0; }
    double fnorm = sqrt(nbo_dot_c(Ex, Ey, Ez, n, f, f));
    double rho_old = 1.0;
    double rho = nbo_dot_c(Ex, Ey, Ez, n, r, z);
    double rr = nbo_dot_c(Ex, Ey, Ez, n, r, r);
    if (rr_hist) rr_hist[0] = rr;
    for (int it = 1; it <= maxit; it++) {
        if (rho == 0.0) break;
        if (tol > 0.0 && sqrt(rr) / fnorm <= tol) break;
        double beta = (it == 1) ? 0.0 : rho / rho_old;
        for (long q = 0; q < npts; q++) p[q] = z[q] + beta * p[q];
        nbo_apply_A(Ex, Ey, Ez, n, D, gxyz, mask, p, w);
        double pap = nbo_dot_c(Ex, Ey, Ez, n, w, p);
        if (!(pap > 0.0) || !isfinite(pap)) { status = 1; break; }
        double alpha = rho / pap;
        for (long q = 0; q < npts; q++) {
            x[q] = x[q] + alpha * p[q];
            r[q] = r[q] - alpha * w[q];
            z[q] = minv[q] * r[q];
        }
        rho_old = rho;
        rho = nbo_dot_c(Ex, Ey, Ez, n, r, z);
        rr = nbo_dot_c(Ex, Ey, Ez, n, r, r);
        iters = it;
        if (rr_hist) rr_hist[it] = rr;
    }
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = fnorm > 0.0 ? sqrt(rr) / fnorm : 0.0;
    free(r); free(z); free(p); free(w);
    return status;
}
