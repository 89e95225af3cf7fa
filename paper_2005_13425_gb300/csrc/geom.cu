// Set-up of the synthetic Nekbone box problem: GLL nodes and weights, the
// derivative matrix, and the geometric factors gxyz of a perturbed box mesh
// (arXiv 2005.13425 Sec. III: SEM Poisson on a cubic domain; Sec. III.A:
// n GLL points per direction; Listing 1: dxm1 and gxyz(.,1..6)).
#include <math.h>

#include "internal.cuh"

namespace nekgb {

// Legendre P_m(x) for m = N-1, N, N+1 by the three-term recurrence.
static void legendre3(int N, double x, double *pm1, double *p0, double *pp1) {
    double a = 1.0, b = x;   // P_0, P_1
    if (N == 0) { *pm1 = 0.0; *p0 = 1.0; *pp1 = x; return; }
    double prev = a;
    for (int k = 1; k <= N; k++) {   // after step k: a = P_k, b = P_{k+1}
        double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
        prev = a;
        a = b;
        b = c;
    }
    *pm1 = prev; *p0 = a; *pp1 = b;
}

// The n = N+1 GLL points are the roots of q(x) = P_{N+1}(x) - P_{N-1}(x),
// which is proportional to (1 - x^2) P_N'(x); q'(x) = (2N+1) P_N(x).
// Newton from the Chebyshev-Gauss-Lobatto points; w_i = 2/(N(N+1)P_N^2).
nb_status host_gll(int n, double *xi, double *w) {
    if (n < 2 || n > kMaxN) return fail(NB_ERR_ARG, "n must be in 2..16");
    const int N = n - 1;
    for (int i = 0; i < n; i++) {
        double x = -cos(M_PI * i / N);
        if (i > 0 && i < N) {
            for (int it = 0; it < 50; it++) {
                double pm1, p0, pp1;
                legendre3(N, x, &pm1, &p0, &pp1);
                double dx = (pp1 - pm1) / ((2 * N + 1) * p0);
                x -= dx;
                if (fabs(dx) < 1e-17) break;
            }
        }
        if (i > 0 && i < N && 2 * i == N) x = 0.0;
        xi[i] = x;
    }
    // symmetrise: the rule is symmetric about 0
    for (int i = 0; i < n / 2; i++) {
        double a = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -a;
        xi[N - i] = a;
    }
    for (int i = 0; i < n; i++) {
        double pm1, p0, pp1;
        legendre3(N, xi[i], &pm1, &p0, &pp1);
        w[i] = 2.0 / ((double)N * (N + 1) * p0 * p0);
    }
    return NB_OK;
}

// Lagrange derivative matrix from barycentric weights:
// D(i,l) = (lam_l / lam_i) / (x_i - x_l), D(i,i) = -sum_{l != i} D(i,l).
nb_status host_dmat(int n, const double *x, double *D) {
    double lam[kMaxN];
    for (int j = 0; j < n; j++) {
        double p = 1.0;
        for (int k = 0; k < n; k++)
            if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < n; i++) {
        double diag = 0.0;
        for (int l = 0; l < n; l++) {
            if (l == i) continue;
            double v = (lam[l] / lam[i]) / (x[i] - x[l]);
            D[i * n + l] = v;
            diag -= v;
        }
        D[i * n + i] = diag;
    }
    return NB_OK;
}

__device__ __forceinline__ void store_g(double *dst, double v) { *dst = v; }
// pairs (hi, lo) for the double-float operator, unscaled
__device__ __forceinline__ void store_g(float2 *dst, double v) {
    const float h = __double2float_rn(v);
    *dst = make_float2(h, __double2float_rn(v - (double)h));
}

struct GeomParams {
    double xi[kMaxN], w[kMaxN], D[kMaxN * kMaxN];
    double amp, s[3];
    int ez0, ez_total;   // the mesh's elements are layers ez0.. of a box ez_total elements high
};

// A context's place in the z direction of its box (a slab of a partitioned
// box starts at layer slab_z0 of slab_ez_global; a whole box at 0 of m.ez).
static void z_extent(const nb_ctx *c, GeomParams &gp) {
    gp.ez0 = c->slab ? c->slab_z0 : 0;
    gp.ez_total = c->slab ? c->slab_ez_global : c->m.ez;
}

// One CTA per element (grid-stride).  Nodal coordinates are the affine box
// position plus amp*s_d*sin(pi X) sin(pi Y) sin(pi Z); the Jacobian applies
// D to the nodal coordinates along r, s and t (isoparametric mapping).
template <typename OutT>
__global__ void box_geometry_kernel(OutT *__restrict__ gxyz, Mesh m, GeomParams gp,
                                    int *__restrict__ bad) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    __shared__ double X[kMaxN], Y[kMaxN], Z[kMaxN], SX[kMaxN], SY[kMaxN], SZ[kMaxN];
    for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
        const int ex = (int)(e % m.ex), ey = (int)((e / m.ex) % m.ey),
                  ez = (int)(e / ((int64_t)m.ex * m.ey));
        __syncthreads();
        if (threadIdx.x < n) {
            const int a = threadIdx.x;
            X[a] = (ex + 0.5 * (gp.xi[a] + 1.0)) / m.ex;
            Y[a] = (ey + 0.5 * (gp.xi[a] + 1.0)) / m.ey;
            Z[a] = (ez + gp.ez0 + 0.5 * (gp.xi[a] + 1.0)) / gp.ez_total;
            SX[a] = sin(M_PI * X[a]);
            SY[a] = sin(M_PI * Y[a]);
            SZ[a] = sin(M_PI * Z[a]);
        }
        __syncthreads();
        for (int p = threadIdx.x; p < n3; p += blockDim.x) {
            const int i = p % n, j = (p / n) % n, k = p / (n * n);
            double J[3][3];
            for (int a = 0; a < 3; a++) {
                double dr = 0.0, ds = 0.0, dt = 0.0;
                const double as = gp.amp * gp.s[a];
                for (int l = 0; l < n; l++) {
                    // x_a at (l,j,k), (i,l,k) and (i,j,l)
                    const double base_r = a == 0 ? X[l] : (a == 1 ? Y[j] : Z[k]);
                    const double base_s = a == 0 ? X[i] : (a == 1 ? Y[l] : Z[k]);
                    const double base_t = a == 0 ? X[i] : (a == 1 ? Y[j] : Z[l]);
                    const double xr = base_r + as * (SX[l] * SY[j] * SZ[k]);
                    const double xs = base_s + as * (SX[i] * SY[l] * SZ[k]);
                    const double xt = base_t + as * (SX[i] * SY[j] * SZ[l]);
                    dr = fma(gp.D[i * n + l], xr, dr);
                    ds = fma(gp.D[j * n + l], xs, ds);
                    dt = fma(gp.D[k * n + l], xt, dt);
                }
                J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
            }
            // cofactors C[a][b] of J; J^{-1} = C^T / det
            double C[3][3];
            C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
            if (!(det > 0.0)) atomicExch(bad, 1);
            // G = J^{-1} J^{-T} = C^T C / det^2; gxyz = w w w det G = w w w C^T C / det
            const double sc = gp.w[i] * gp.w[j] * gp.w[k] / det;
            double G[6];
            const int bb[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
            for (int q = 0; q < 6; q++) {
                const int b = bb[q], c = cc[q];
                G[q] = (C[0][b] * C[0][c] + C[1][b] * C[1][c] + C[2][b] * C[2][c]) * sc;
            }
            OutT *g = gxyz + e * 6 * n3 + p;
            for (int q = 0; q < 6; q++) store_g(g + q * n3, G[q]);
        }
    }
}

// Nodal coordinates xyz[E][3][n^3] of the perturbed box (same map as above).
__global__ void box_coords_kernel(double *__restrict__ xyz, Mesh m, GeomParams gp) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const int ex = (int)(e % m.ex), ey = (int)((e / m.ex) % m.ey), ez = (int)(e / ((int64_t)m.ex * m.ey));
        const double X = (ex + 0.5 * (gp.xi[i] + 1.0)) / m.ex;
        const double Y = (ey + 0.5 * (gp.xi[j] + 1.0)) / m.ey;
        const double Z = (ez + gp.ez0 + 0.5 * (gp.xi[k] + 1.0)) / gp.ez_total;
        const double bump = sin(M_PI * X) * sin(M_PI * Y) * sin(M_PI * Z);
        double *o = xyz + e * 3 * n3 + p;
        o[0] = X + gp.amp * gp.s[0] * bump;
        o[n3] = Y + gp.amp * gp.s[1] * bump;
        o[2 * n3] = Z + gp.amp * gp.s[2] * bump;
    }
}

nb_status launch_box_coords(nb_ctx *c, double *xyz) {
    if (!c->is_box) return fail(NB_ERR_STATE, "coordinates are known only for nb_setup_box contexts");
    GeomParams gp;
    nb_status st = host_gll(c->m.n, gp.xi, gp.w);
    if (st != NB_OK) return st;
    gp.amp = c->box_amp;
    gp.s[0] = c->box_s[0]; gp.s[1] = c->box_s[1]; gp.s[2] = c->box_s[2];
    z_extent(c, gp);
    const int sms = device_sms();
    box_coords_kernel<<<grid_blocks(c->m.npts, 256, sms * 8), 256, 0, c->stream>>>(xyz, c->m, gp);
    NB_LAUNCH_CHECK("box_coords_kernel");
    return NB_OK;
}

nb_status launch_box_geometry(nb_ctx *c, double amp, const double *s, int *bad_dev) {
    GeomParams gp;
    const int n = c->m.n;
    nb_status st = host_gll(n, gp.xi, gp.w);
    if (st != NB_OK) return st;
    for (int q = 0; q < n * n; q++) gp.D[q] = c->D_host[q];
    gp.amp = amp;
    gp.s[0] = s[0]; gp.s[1] = s[1]; gp.s[2] = s[2];
    z_extent(c, gp);
    const int sms = device_sms();
    const int grid = (int)(c->m.E < (int64_t)sms * 8 ? c->m.E : (int64_t)sms * 8);
    box_geometry_kernel<double><<<grid, 256, 0, c->stream>>>(c->d_gxyz, c->m, gp, bad_dev);
    NB_LAUNCH_CHECK("box_geometry_kernel");
    return NB_OK;
}

// Geometric factors of a perturbed box as (hi, lo) float pairs (no scaling),
// for problems of the batched engine; D is the context-free GLL matrix.
nb_status launch_box_geometry_pairs(const Mesh &m, double amp, const double *s, const double *D,
                                    float2 *out, int *bad_dev, cudaStream_t stream) {
    GeomParams gp;
    nb_status st = host_gll(m.n, gp.xi, gp.w);
    if (st != NB_OK) return st;
    for (int q = 0; q < m.n * m.n; q++) gp.D[q] = D[q];
    gp.amp = amp;
    gp.s[0] = s[0]; gp.s[1] = s[1]; gp.s[2] = s[2];
    gp.ez0 = 0;
    gp.ez_total = m.ez;
    const int sms = device_sms();
    const int grid = (int)(m.E < (int64_t)sms * 8 ? m.E : (int64_t)sms * 8);
    box_geometry_kernel<float2><<<grid, 256, 0, stream>>>(out, m, gp, bad_dev);
    NB_LAUNCH_CHECK("box_geometry_kernel<pairs>");
    return NB_OK;
}

}  // namespace nekgb
