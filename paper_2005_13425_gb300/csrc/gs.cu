// Direct stiffness summation (dssum), Dirichlet mask and the index work
// behind them, for the structured box mesh (arXiv 2005.13425 Sec. III: the
// second step of Ax communicates the element results to the neighbouring
// elements; Sec. VI.B: masking of the boundary conditions).
//
// dssum is a pull over unique nodes: only nodes on element interfaces have
// more than one copy, and their set is enumerated directly (no tables are
// read), so the kernel moves just the interface values.  Each node adds its
// copies from +0.0 in ascending element order and writes the sum back to
// every copy, which makes the result bit-for-bit independent of the launch.
#include "internal.cuh"

namespace nekgb {

// Non-plane coordinate q (of NX - (Ex - 1)) -> global coordinate: 0, the
// element-interior indices, and the last node.
__device__ __forceinline__ int64_t nonplane_coord(int64_t q, int ne, int n, int64_t NG) {
    if (q == 0) return 0;
    const int64_t last = (int64_t)ne * (n - 2) + 1;
    if (q == last) return NG - 1;
    const int64_t qq = q - 1;
    return (qq / (n - 2)) * (n - 1) + 1 + qq % (n - 2);
}

// Copies of global coordinate g along one direction: up to two (element,
// local index) pairs, in ascending element order.
__device__ __forceinline__ int copies_1d(int64_t g, int ne, int n, int *el, int *li) {
    const int64_t a = g / (n - 1);
    const int64_t rem = g - a * (n - 1);
    if (rem == 0 && a > 0 && a < ne) {
        el[0] = (int)a - 1; li[0] = n - 1;
        el[1] = (int)a;     li[1] = 0;
        return 2;
    }
    const int64_t ee = a < ne ? a : ne - 1;
    el[0] = (int)ee;
    li[0] = (int)(g - ee * (n - 1));
    return 1;
}

__global__ void dssum_kernel(double *__restrict__ w, Mesh m, int64_t cx, int64_t cy, int64_t cz,
                             const CgScalars *__restrict__ sc) {
    if (sc && sc->done) return;
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t total = cx + cy + cz;
    const int64_t NXp = m.NX - (m.ex - 1), NYp = m.NY - (m.ey - 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t gx, gy, gz;
        if (q < cx) {              // interior x-planes, all y, z
            int64_t r = q;
            gy = r % m.NY; r /= m.NY;
            gz = r % m.NZ; r /= m.NZ;
            gx = (r + 1) * (n - 1);
        } else if (q < cx + cy) {  // interior y-planes, x off the x-planes
            int64_t r = q - cx;
            gx = nonplane_coord(r % NXp, m.ex, n, m.NX); r /= NXp;
            gz = r % m.NZ; r /= m.NZ;
            gy = (r + 1) * (n - 1);
        } else {                   // interior z-planes, x and y off the planes
            int64_t r = q - cx - cy;
            gx = nonplane_coord(r % NXp, m.ex, n, m.NX); r /= NXp;
            gy = nonplane_coord(r % NYp, m.ey, n, m.NY); r /= NYp;
            gz = (r + 1) * (n - 1);
        }
        int elx[2], lix[2], ely[2], liy[2], elz[2], liz[2];
        const int nx = copies_1d(gx, m.ex, n, elx, lix);
        const int ny = copies_1d(gy, m.ey, n, ely, liy);
        const int nz = copies_1d(gz, m.ez, n, elz, liz);
        int64_t idx[8];
        int c = 0;
        for (int a = 0; a < nz; a++)
            for (int b = 0; b < ny; b++)
                for (int d = 0; d < nx; d++) {
                    const int64_t e = elx[d] + (int64_t)m.ex * (ely[b] + (int64_t)m.ey * elz[a]);
                    idx[c++] = e * n3 + lix[d] + n * (liy[b] + (int64_t)n * liz[a]);
                }
        double s = 0.0;
        for (int k = 0; k < c; k++) s = __dadd_rn(s, w[idx[k]]);
        for (int k = 0; k < c; k++) w[idx[k]] = s;
    }
}

// Mask: w := +0.0 at Dirichlet points.  Box mask: points whose global node
// lies on a face of the box; otherwise the context's mask array.
__global__ void mask_kernel(double *__restrict__ w, Mesh m, const uint8_t *__restrict__ mask,
                            const CgScalars *__restrict__ sc) {
    if (sc && sc->done) return;
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        bool zero;
        if (mask) {
            zero = mask[q] == 0;
        } else {
            const int64_t e = q / n3;
            const int p = (int)(q - e * n3);
            const int i = p % n, j = (p / n) % n, k = p / (n * n);
            const int ex = (int)(e % m.ex), ey = (int)((e / m.ex) % m.ey), ez = (int)(e / ((int64_t)m.ex * m.ey));
            zero = (i == 0 && ex == 0) || (i == n - 1 && ex == m.ex - 1) ||
                   (j == 0 && ey == 0) || (j == n - 1 && ey == m.ey - 1) ||
                   (k == 0 && ez == 0) || (k == n - 1 && ez == m.ez - 1);
        }
        if (zero) w[q] = 0.0;
    }
}

__global__ void scatter_unique_kernel(const double *__restrict__ g, double *__restrict__ loc, Mesh m) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const int64_t ex = e % m.ex, ey = (e / m.ex) % m.ey, ez = e / ((int64_t)m.ex * m.ey);
        const int64_t gx = ex * (n - 1) + i, gy = ey * (n - 1) + j, gz = ez * (n - 1) + k;
        loc[q] = g[gx + m.NX * (gy + m.NY * gz)];
    }
}

__global__ void tables_kernel(int64_t *__restrict__ gid, int32_t *__restrict__ mult,
                              uint8_t *__restrict__ maskout, const uint8_t *__restrict__ mask, Mesh m) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const int ex = (int)(e % m.ex), ey = (int)((e / m.ex) % m.ey), ez = (int)(e / ((int64_t)m.ex * m.ey));
        const int64_t gx = (int64_t)ex * (n - 1) + i, gy = (int64_t)ey * (n - 1) + j,
                      gz = (int64_t)ez * (n - 1) + k;
        if (gid) gid[q] = gx + m.NX * (gy + m.NY * gz);
        if (mult) mult[q] = mult_1d(i, ex, m.ex, n) * mult_1d(j, ey, m.ey, n) * mult_1d(k, ez, m.ez, n);
        if (maskout) {
            if (mask) {
                maskout[q] = mask[q] ? 1 : 0;
            } else {
                const bool b = gx == 0 || gx == m.NX - 1 || gy == 0 || gy == m.NY - 1 ||
                               gz == 0 || gz == m.NZ - 1;
                maskout[q] = b ? 0 : 1;
            }
        }
    }
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

nb_status launch_dssum_sc(nb_ctx *c, double *w, const CgScalars *sc) {
    const Mesh &m = c->m;
    const int64_t NXp = m.NX - (m.ex - 1), NYp = m.NY - (m.ey - 1);
    const int64_t cx = (int64_t)(m.ex - 1) * m.NY * m.NZ;
    const int64_t cy = (int64_t)(m.ey - 1) * NXp * m.NZ;
    const int64_t cz = (int64_t)(m.ez - 1) * NXp * NYp;
    const int64_t total = cx + cy + cz;
    if (total == 0) return NB_OK;
    const int threads = 256;
    const int grid = grid_blocks(total, threads, sm_count() * 8);
    LaunchTimer tm(c, NB_K_DSSUM);
    dssum_kernel<<<grid, threads, 0, c->stream>>>(w, m, cx, cy, cz, sc);
    NB_LAUNCH_CHECK("dssum_kernel");
    return NB_OK;
}

nb_status launch_mask_sc(nb_ctx *c, double *w, const CgScalars *sc) {
    const int threads = 256;
    const int grid = grid_blocks(c->m.npts, threads, sm_count() * 8);
    LaunchTimer tm(c, NB_K_MASK);
    mask_kernel<<<grid, threads, 0, c->stream>>>(w, c->m, c->d_mask, sc);
    NB_LAUNCH_CHECK("mask_kernel");
    return NB_OK;
}

nb_status launch_dssum(nb_ctx *c, double *w, bool with_mask) {
    nb_status s = launch_dssum_sc(c, w, nullptr);
    if (s != NB_OK || !with_mask) return s;
    return launch_mask_sc(c, w, nullptr);
}

nb_status launch_mask(nb_ctx *c, double *w) { return launch_mask_sc(c, w, nullptr); }

nb_status launch_scatter_unique(nb_ctx *c, const double *g, double *loc) {
    const int threads = 256;
    const int grid = grid_blocks(c->m.npts, threads, sm_count() * 8);
    LaunchTimer tm(c, NB_K_OTHER);
    scatter_unique_kernel<<<grid, threads, 0, c->stream>>>(g, loc, c->m);
    NB_LAUNCH_CHECK("scatter_unique_kernel");
    return NB_OK;
}

nb_status launch_tables(nb_ctx *c, int64_t *gid, int32_t *mult, uint8_t *mask) {
    if (!gid && !mult && !mask) return NB_OK;
    const int threads = 256;
    const int grid = grid_blocks(c->m.npts, threads, sm_count() * 8);
    LaunchTimer tm(c, NB_K_OTHER);
    tables_kernel<<<grid, threads, 0, c->stream>>>(gid, mult, mask, c->d_mask, c->m);
    NB_LAUNCH_CHECK("tables_kernel");
    return NB_OK;
}

}  // namespace nekgb
