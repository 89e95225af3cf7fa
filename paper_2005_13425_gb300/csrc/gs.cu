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
#include <type_traits>

#include "df.cuh"
#include "gs_fast.cuh"
#include "gs_nodes.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

// Plain dssum (CG = false) or the fused solver step (CG = true), over the
// shared nodes grouped by category (faces, edges, vertices; DsCat): each
// node adds its copies from +0.0 in ascending element order and writes the
// sum back to every copy.  In the solver the ax_e head has already summed
// <w,p>_c as local products (p is continuous, so the assembled product
// equals the sum of the unassembled ones); the last CTA here reduces those
// partials, forms alpha = rho/<w,p>_c and flags a breakdown.  N is the
// number of points per direction.
template <typename T, bool CG, int N>
__global__ void __launch_bounds__(256, 5)
dssum_kernel(T *__restrict__ w, DsCat dd, CgScalars *sc, double *partials, int slot0) {
    if (sc && sc->done) return;
    const int total = dd.o[7];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int64_t idx[8];
        const int c = cat_copies<N>(q, dd, idx);
        // (+0.0) + v equals v except for v = -0.0, so the first add is a sign
        // fix-up done with integer operations; the remaining adds are
        // exact-count loops (no predicated-off FP64 adds on GB300's narrow
        // FP64 pipe).
        if (c == 2) {
            const T s = plus_zero(w[idx[0]]) + w[idx[1]];
            w[idx[0]] = s;
            w[idx[1]] = s;
        } else if (c == 4) {
            T a[4];
#pragma unroll
            for (int k = 0; k < 4; k++) a[k] = w[idx[k]];
            T s = plus_zero(a[0]);
#pragma unroll
            for (int k = 1; k < 4; k++) s = s + a[k];
#pragma unroll
            for (int k = 0; k < 4; k++) w[idx[k]] = s;
        } else {
            T a[8];
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = w[idx[k]];
            T s = plus_zero(a[0]);
#pragma unroll
            for (int k = 1; k < 8; k++) s = s + a[k];
#pragma unroll
            for (int k = 0; k < 8; k++) w[idx[k]] = s;
        }
    }
    if (CG) {
        double v[1] = {0.0}, tot[1];
        if (!last_block_reduce<1>(v, partials, 0, slot0 + blockIdx.x, slot0 + gridDim.x, gridDim.x,
                                  &sc->ticket, tot))
            return;
        if (threadIdx.x != 0) return;
        const double pap = tot[0];
        sc->pap = pap;
        if (!(pap > 0.0) || !isfinite(pap)) {
            sc->status = (int)NB_ERR_BREAKDOWN;
            sc->done = 1;
            sc->x_alpha = 0.0;
        } else {
            sc->alpha = sc->rho / pap;
            sc->x_alpha = sc->alpha;
        }
    }
}

// Box mask: zero every local point on a face of the box (only those points
// are visited: two faces per direction, n^2 points per face element).
__global__ void mask_box_kernel(double *__restrict__ w, Mesh m, const CgScalars *__restrict__ sc) {
    if (sc && sc->done) return;
    const int n = m.n, n2 = n * n;
    const int64_t n3 = (int64_t)n * n * n;
    const int fx = m.ey * m.ez * n2, fy = m.ex * m.ez * n2, fz = m.ex * m.ey * n2;
    const int total = 2 * (fx + fy + fz);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int ex, ey, ez, i, j, k, r;
        if (q < 2 * fx) {
            const int side = q / fx;
            r = q - side * fx;
            const int pt = r % n2, el = r / n2;
            ey = el % m.ey; ez = el / m.ey; ex = side ? m.ex - 1 : 0;
            j = pt % n; k = pt / n; i = side ? n - 1 : 0;
        } else if (q < 2 * (fx + fy)) {
            const int qq = q - 2 * fx;
            const int side = qq / fy;
            r = qq - side * fy;
            const int pt = r % n2, el = r / n2;
            ex = el % m.ex; ez = el / m.ex; ey = side ? m.ey - 1 : 0;
            i = pt % n; k = pt / n; j = side ? n - 1 : 0;
        } else {
            const int qq = q - 2 * (fx + fy);
            const int side = qq / fz;
            r = qq - side * fz;
            const int pt = r % n2, el = r / n2;
            ex = el % m.ex; ey = el / m.ex; ez = side ? m.ez - 1 : 0;
            i = pt % n; j = pt / n; k = side ? n - 1 : 0;
        }
        const int64_t e = ex + (int64_t)m.ex * (ey + (int64_t)m.ey * ez);
        w[e * n3 + i + n * (j + n * k)] = 0.0;
    }
}

// Mask from the context's array: w := +0.0 where mask == 0.
__global__ void mask_array_kernel(double *__restrict__ w, Mesh m, const uint8_t *__restrict__ mask,
                                  const CgScalars *__restrict__ sc) {
    if (sc && sc->done) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x)
        if (mask[q] == 0) w[q] = 0.0;
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


static int sm_count() { return device_sms(); }


// One wave of CTAs (five per SM, the kernel's register bound) striding over
// the shared nodes (one block reduction per CTA in the solver step).
int dssum_grid(const nb_ctx *c) {
    int cx, cy, cz;
    shared_counts(c->m, cx, cy, cz);
    return grid_blocks((int64_t)cx + cy + cz, 256, sm_count() * 5);
}

template <typename T, bool CG>
static void dssum_launch(nb_ctx *c, T *w, CgScalars *sc, double *partials, int slot0) {
    const DsCat dd = make_ds_cat(c->m);
    const int grid = dssum_grid(c);
    switch (c->m.n) {
#define NB_CASE(NN) \
    case NN: dssum_kernel<T, CG, NN><<<grid, 256, 0, c->stream>>>(w, dd, sc, partials, slot0); break;
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
        default: break;
    }
}

nb_status launch_dssum_sc(nb_ctx *c, double *w, const CgScalars *sc) {
    int cx, cy, cz;
    shared_counts(c->m, cx, cy, cz);
    if ((int64_t)cx + cy + cz == 0) return NB_OK;
    LaunchTimer tm(c, NB_K_DSSUM);
    dssum_launch<double, false>(c, w, const_cast<CgScalars *>(sc), nullptr, 0);
    NB_LAUNCH_CHECK("dssum_kernel");
    return NB_OK;
}

// Fused solver step: dssum of w and alpha = rho/<w,p>_c.
nb_status launch_dssum_cg(nb_ctx *c) {
    LaunchTimer tm(c, NB_K_DSSUM);
    dssum_launch<double, true>(c, c->d_w, c->d_sc, c->d_partials, c->ax_grid);
    NB_LAUNCH_CHECK("dssum_kernel<cg>");
    return NB_OK;
}

// Plain FP32 dssum (tests of the inner operator).
nb_status launch_dssum32(nb_ctx *c, float *w) {
    int cx, cy, cz;
    shared_counts(c->m, cx, cy, cz);
    if ((int64_t)cx + cy + cz == 0) return NB_OK;
    LaunchTimer tm(c, NB_K_DSSUM);
    dssum_launch<float, false>(c, w, nullptr, nullptr, 0);
    NB_LAUNCH_CHECK("dssum_kernel<f32>");
    return NB_OK;
}

nb_status launch_mask_sc(nb_ctx *c, double *w, const CgScalars *sc) {
    const int threads = 256;
    LaunchTimer tm(c, NB_K_MASK);
    if (c->d_mask) {
        const int grid = grid_blocks(c->m.npts, threads, sm_count() * 8);
        mask_array_kernel<<<grid, threads, 0, c->stream>>>(w, c->m, c->d_mask, sc);
    } else {
        const Mesh &m = c->m;
        const int64_t total = 2 * (int64_t)m.n * m.n * ((int64_t)m.ey * m.ez + (int64_t)m.ex * m.ez +
                                                        (int64_t)m.ex * m.ey);
        const int grid = grid_blocks(total, threads, sm_count() * 8);
        mask_box_kernel<<<grid, threads, 0, c->stream>>>(w, c->m, sc);
    }
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
