// ax_e in native FP64: the element-local Poisson operator of Listing 1
// (arXiv 2005.13425, Sec. III) evaluated layer by layer.
//
// One CTA owns one element at a time (grid-stride over elements) with one
// thread per (i,j) column of the element.  The element's u is staged in
// shared memory; each thread keeps its w(i,j,:) column in registers.  For
// every layer k the thread forms wr, ws (from shared memory) and wt (from
// the staged column), contracts them with the six geometric factors, and
// the layer's ur/us go through shared memory for the transposed r/s sums
// while ut is scattered into the register column (the t-direction of the
// transposed derivative).  This keeps Listing 1's arithmetic: each output is
// sum_l dxtm1 * (ur, us, ut), with FP64 fused multiply-adds.
//
// GB300 executes FP64 at ~1 TFLOP/s (measured), so this kernel is bound by
// the FP64 pipe, not by HBM; the double-float kernel (ax_df.cu) is the fast
// FP64-accurate path.  This one is kept as the plain-arithmetic variant.
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

template <int N>
struct AxFp64Smem {
    double D[N * N];   // D[i*N+l] = dxm1(i,l)
    double u[N * N * N];
    double ur[2][N * N];
    double us[2][N * N];
};

struct AxCgArgs {
    const double *r;      // residual
    double *p;            // search direction, updated in place
    double *x;            // iterate, receives the owed x += x_alpha p
    const double *minv;   // Jacobi inverse diagonal (z = minv r) or null
    const CgScalars *sc;
    double *partials;     // fused: one <w,p> partial per CTA
    int fuse;             // zero box-face points and sum the local products w p
    Mesh m;
};

// MODE 0: w = ax_e(u).
// MODE 1: CG iteration head: x += x_alpha p, p = r + beta p (written back),
//         w = ax_e(p); when fused, box-face points of w are zeroed and the
//         local products w p (whose sum is <w,p>_c after assembly, p being
//         continuous) are reduced per CTA.
template <int N, int MODE>
__global__ void __launch_bounds__(((N * N + 31) / 32) * 32)
ax_fp64_kernel(const double *__restrict__ u, double *__restrict__ w,
               const double *__restrict__ gxyz, const double *__restrict__ Dg, int64_t E,
               AxCgArgs cg) {
    constexpr int N2 = N * N, N3 = N * N * N;
    __shared__ AxFp64Smem<N> sm;
    __shared__ double red[32];
    double beta = 0.0, xa = 0.0, dot = 0.0;
    if (MODE == 1) {
        if (cg.sc->done) return;
        beta = cg.sc->it == 0 ? 0.0 : cg.sc->beta;
        xa = cg.sc->x_alpha;
    }
    const int t = threadIdx.x;
    const bool act = t < N2;
    // Threads past N*N (when N*N is not a multiple of 32) run the same code
    // on a clamped column and store nothing, so every barrier is reached by
    // the whole CTA.
    const int tc = act ? t : N2 - 1;
    const int i = tc % N, j = tc / N;
    for (int q = t; q < N2; q += blockDim.x) sm.D[q] = Dg[q];

    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int64_t base = e * N3;
        __syncthreads();   // previous element fully consumed
        for (int q = t; q < N3; q += blockDim.x) {
            double v;
            if (MODE == 1) {
                const double pold = cg.p[base + q];
                if (xa != 0.0) cg.x[base + q] = fma(xa, pold, cg.x[base + q]);
                const double z = cg.minv ? cg.r[base + q] * cg.minv[base + q] : cg.r[base + q];
                v = fma(beta, pold, z);
                cg.p[base + q] = v;
            } else {
                v = __ldg(u + base + q);
            }
            sm.u[q] = v;
        }
        __syncthreads();
        double ucol[N], wcol[N];
#pragma unroll
        for (int l = 0; l < N; l++) {
            ucol[l] = sm.u[i + N * (j + N * l)];
            wcol[l] = 0.0;
        }
        const double *g = gxyz + e * 6 * N3 + j * N + i;
#pragma unroll
        for (int k = 0; k < N; k++) {
            const int buf = k & 1;
            double wr = 0.0, ws = 0.0, wt = 0.0;
#pragma unroll
            for (int l = 0; l < N; l++) {
                wr = fma(sm.D[i * N + l], sm.u[l + N * (j + N * k)], wr);
                ws = fma(sm.D[j * N + l], sm.u[i + N * (l + N * k)], ws);
                wt = fma(sm.D[k * N + l], ucol[l], wt);
            }
            const int off = k * N2;
            const double g0 = __ldg(g + 0 * N3 + off), g1 = __ldg(g + 1 * N3 + off);
            const double g2 = __ldg(g + 2 * N3 + off), g3 = __ldg(g + 3 * N3 + off);
            const double g4 = __ldg(g + 4 * N3 + off), g5 = __ldg(g + 5 * N3 + off);
            const double ur = fma(g0, wr, fma(g1, ws, g2 * wt));
            const double us = fma(g1, wr, fma(g3, ws, g4 * wt));
            const double ut = fma(g2, wr, fma(g4, ws, g5 * wt));
            if (act) {
                sm.ur[buf][j * N + i] = ur;
                sm.us[buf][j * N + i] = us;
            }
            // t-direction of the transposed derivative:
            // w(i,j,m) += dxtm1(m,k) ut(i,j,k) = D(k,m) ut(i,j,k)
#pragma unroll
            for (int m = 0; m < N; m++) wcol[m] = fma(sm.D[k * N + m], ut, wcol[m]);
            // ur/us of this layer complete; double buffering lets the next
            // layer write the other buffer without a second barrier.
            __syncthreads();
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < N; l++) {
                acc = fma(sm.D[l * N + i], sm.ur[buf][j * N + l], acc);
                acc = fma(sm.D[l * N + j], sm.us[buf][l * N + i], acc);
            }
            wcol[k] += acc;
        }
        if (act) {
            int ex = 0, ey = 0, ez = 0;
            if (MODE == 1) element_coords(e, cg.m, ex, ey, ez);
#pragma unroll
            for (int m = 0; m < N; m++) {
                double wv = wcol[m];
                if (MODE == 1 && cg.fuse) {
                    if (on_box_face(i, j, m, ex, ey, ez, cg.m))
                        wv = 0.0;
                    else
                        dot = fma(wv, cg.p[base + i + N * (j + N * m)], dot);
                }
                w[base + i + N * (j + N * m)] = wv;
            }
        }
    }
    if (MODE == 1 && cg.fuse) {
        const double b = block_sum(dot, red);
        if (t == 0) cg.partials[blockIdx.x] = b;
    }
}

template <int N>
static nb_status launch_n(nb_ctx *c, const double *u, double *w, int mode) {
    const int threads = ((N * N + 31) / 32) * 32;
    int occ = 0;
    const int sms = device_sms();
    if (mode == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ax_fp64_kernel<N, 0>, threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ax_fp64_kernel<N, 1>, threads, 0);
    if (occ < 1) occ = 1;
    const int64_t cap = (int64_t)sms * occ;
    const int grid = (int)(c->m.E < cap ? c->m.E : cap);
    AxCgArgs cg{};
    cg.m = c->m;
    LaunchTimer tm(c, NB_K_AX);
    if (mode == 0) {
        ax_fp64_kernel<N, 0><<<grid, threads, 0, c->stream>>>(u, w, c->d_gxyz, c->d_D, c->m.E, cg);
    } else {
        cg.r = c->d_r;
        cg.p = c->d_p;
        cg.x = c->d_x;
        cg.minv = c->d_minv;
        cg.sc = c->d_sc;
        cg.partials = c->d_partials;
        cg.fuse = c->fused_cg ? 1 : 0;
        c->ax_grid = grid;
        ax_fp64_kernel<N, 1><<<grid, threads, 0, c->stream>>>(nullptr, c->d_w, c->d_gxyz, c->d_D,
                                                              c->m.E, cg);
    }
    NB_LAUNCH_CHECK("ax_fp64_kernel");
    return NB_OK;
}

nb_status launch_ax_fp64(nb_ctx *c, const double *u, double *w, int mode) {
    switch (c->m.n) {
#define NB_CASE(NN) case NN: return launch_n<NN>(c, u, w, mode);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
}

}  // namespace nekgb
