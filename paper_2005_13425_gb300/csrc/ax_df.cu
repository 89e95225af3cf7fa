// ax_e in double-float arithmetic on the FP32 pipes: the element-local
// Poisson operator of Listing 1 (arXiv 2005.13425, Sec. III) to FP64
// accuracy on GB300, whose FP64 pipe delivers only ~1 TFLOP/s.
//
// Arithmetic.  u, gxyz and D are split into pairs of floats (48-bit
// significands).  Every contraction -- the forward derivatives wr, ws, wt,
// the 3x3 geometric contraction and the transposed derivatives -- is a
// compensated dot product (TwoProd + TwoSum, Dot2), and the three
// transposed-derivative partial sums are added as pairs.  Inputs are scaled
// by exact powers of two (per element for u, once per context for gxyz) so
// the pairs keep their full relative precision whatever the data's
// magnitude; the output is scaled back exactly.
//
// Thread layout ("line threads").  A CTA owns one element at a time and has
// 3 n^2 working threads: thread (d, a0, a1) owns one line of the element
// along direction d (r: (j,k); s: (i,k); t: (i,j)).  In the forward phase a
// thread loads its n inputs once from shared memory and produces the n
// derivative values of its line; the entries of D are compile-time indexed
// kernel parameters, so they are constant-bank operands and cost no loads.
// A pointwise phase contracts (wr, ws, wt) with the six geometric factors
// (streamed from HBM, coalesced) into (ur, us, ut) in place.  The backward
// phase is the same line pattern with D^T, each direction writing its own
// partial array, and a final pointwise phase adds the three partials and
// writes w.  Four barriers per element; shared memory holds six n^3 arrays
// of pairs (48 KB at n = 10).
#include <math.h>

#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

template <int N>
struct DfMat {
    float h[N * N];   // h[m*N + l] + l_[m*N + l] = D(m, l)
    float l[N * N];
};

// Even-odd form of a centro-antisymmetric matrix M (M(N-1-m, N-1-l) =
// -M(m,l), which holds for the GLL derivative matrix and its transpose).
// With H = N/2, xs_l = x_l + x_{N-1-l}, xd_l = x_l - x_{N-1-l} (l < H):
//   y_m       = P_m + Q_m,   y_{N-1-m} = P_m - Q_m   (m < H)
//   P_m = sum_{l<H} a(m,l) xd_l,            a(m,l) = (M(m,l) + M(N-1-m,l))/2
//   Q_m = sum_{l<H} b(m,l) xs_l + b(m,H) x_H, b(m,l) = (M(m,l) - M(N-1-m,l))/2
// and for odd N the middle output y_H = sum_{l<H} M(H,l) xd_l + M(H,H) x_H.
// This halves the products of a line (Solomonoff's even-odd decomposition).
template <int N>
struct EoMat {
    static constexpr int H = N / 2;
    float ah[H * H], al[H * H];
    float bh[H * (H + 1)], bl[H * (H + 1)];
    float ch[H + 1], cl[H + 1];
};

template <int N>
struct DfEo {
    EoMat<N> fwd;   // M = D
    EoMat<N> bwd;   // M = D^T
};

struct AxDfArgs {
    const double *u;      // MODE 0 input
    double *w;            // output (FP64, local storage)
    const double *r;      // MODE 1: residual
    double *p;            // MODE 1: search direction, updated in place
    double *x;            // MODE 1: iterate, receives the owed x += x_alpha p
    const CgScalars *sc;  // MODE 1
    double *partials;     // MODE 1 fused: one <w,p> partial per CTA
    int fuse;             // MODE 1: zero box-face points, interior <w,p>
    Mesh m;
    const float2 *g;      // gxyz pairs [E][6][n^3], scaled by 2^-(gexp-1023)
    int gexp;             // biased exponent of max|gxyz|
    int64_t E;
};

// One line task per thread up to n = 12; two per thread above, so that the
// n-long line held in registers does not spill at n = 16.
__host__ __device__ constexpr int ax_df_threads(int n) {
    return n <= 12 ? ((3 * n * n + 31) / 32) * 32 : ((3 * n * n + 1) / 2 + 31) / 32 * 32;
}

// Line task -> (first point, stride) of the line and the direction.
template <int N>
__device__ __forceinline__ int line_of(int task, int &stride) {
    constexpr int N2 = N * N;
    const int d = task / N2;
    const int c = task - d * N2;
    const int a0 = c % N, a1 = c / N;
    if (d == 0) {        // along r: line (j = a0, k = a1)
        stride = 1;
        return N * (a0 + N * a1);
    }
    if (d == 1) {        // along s: line (i = a0, k = a1)
        stride = N;
        return a0 + N2 * a1;
    }
    stride = N2;         // along t: line (i = a0, j = a1)
    return a0 + N * a1;
}

// out(base + m*stride) = sum_l M(m,l) in(base + l*stride), M = D or D^T,
// n compensated dot products of n terms.
template <int N, bool TR>
__device__ __forceinline__ void line_plain(const float2 *in, float2 *out, int base, int stride,
                                           const DfMat<N> &D) {
    float xh[N], xl[N];
#pragma unroll
    for (int l = 0; l < N; l++) {
        const float2 v = in[base + l * stride];
        xh[l] = v.x;
        xl[l] = v.y;
    }
#pragma unroll
    for (int m = 0; m < N; m++) {
        const int i0 = TR ? m : m * N;
        dfa::Acc acc = dfa::first(D.h[i0], D.l[i0], xh[0], xl[0]);
#pragma unroll
        for (int l = 1; l < N; l++) {
            const int il = TR ? l * N + m : m * N + l;
            dfa::fma(acc, D.h[il], D.l[il], xh[l], xl[l]);
        }
        out[base + m * stride] = dfa::norm(acc);
    }
}

// The same line product in even-odd form (see EoMat): pair sums and
// differences, then 2 dot products of N/2 terms per output pair.
template <int N>
__device__ __forceinline__ void line_eo(const float2 *in, float2 *out, int base, int stride,
                                        const EoMat<N> &M) {
    constexpr int H = N / 2;
    float sh[H], sl[H], dh[H], dl[H];
#pragma unroll
    for (int l = 0; l < H; l++) {
        const float2 a = in[base + l * stride], b = in[base + (N - 1 - l) * stride];
        const float2 s = dfa::add(a, b);
        const float2 d = dfa::add(a, make_float2(-b.x, -b.y));
        sh[l] = s.x; sl[l] = s.y;
        dh[l] = d.x; dl[l] = d.y;
    }
    float ch = 0.f, cl = 0.f;
    if (N & 1) {
        const float2 c = in[base + H * stride];
        ch = c.x;
        cl = c.y;
    }
#pragma unroll
    for (int m = 0; m < H; m++) {
        dfa::Acc P = dfa::first(M.ah[m * H], M.al[m * H], dh[0], dl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(P, M.ah[m * H + l], M.al[m * H + l], dh[l], dl[l]);
        dfa::Acc Q = dfa::first(M.bh[m * (H + 1)], M.bl[m * (H + 1)], sh[0], sl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(Q, M.bh[m * (H + 1) + l], M.bl[m * (H + 1) + l], sh[l], sl[l]);
        if (N & 1) dfa::fma(Q, M.bh[m * (H + 1) + H], M.bl[m * (H + 1) + H], ch, cl);
        out[base + m * stride] = dfa::add_acc(P, Q, 1.f);
        out[base + (N - 1 - m) * stride] = dfa::add_acc(P, Q, -1.f);
    }
    if (N & 1) {
        dfa::Acc Y = dfa::first(M.ch[0], M.cl[0], dh[0], dl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(Y, M.ch[l], M.cl[l], dh[l], dl[l]);
        dfa::fma(Y, M.ch[H], M.cl[H], ch, cl);
        out[base + H * stride] = dfa::norm(Y);
    }
}

template <int N, bool EO>
struct DfConsts;
template <int N>
struct DfConsts<N, false> { using type = DfMat<N>; };
template <int N>
struct DfConsts<N, true> { using type = DfEo<N>; };

template <int N, int MODE, bool EO>
__global__ void __launch_bounds__(ax_df_threads(N))
ax_df_kernel(AxDfArgs a, const __grid_constant__ typename DfConsts<N, EO>::type D) {
    constexpr int N2 = N * N, N3 = N * N * N;
    constexpr int T = ax_df_threads(N);
    extern __shared__ float2 sm[];
    float2 *U = sm;            // input pairs; later the r-partial of w
    float2 *W0 = sm + N3;      // wr -> ur
    float2 *W1 = sm + 2 * N3;  // ws -> us
    float2 *W2 = sm + 3 * N3;  // wt -> ut
    float2 *P1 = sm + 4 * N3;  // s-partial of w
    float2 *P2 = sm + 5 * N3;  // t-partial of w
    double *raw = reinterpret_cast<double *>(U);
    __shared__ int s_emax;

    __shared__ double red[32];
    double beta = 0.0, xa = 0.0, dot = 0.0;
    if (MODE == 1) {
        if (a.sc->done) return;
        beta = a.sc->it == 0 ? 0.0 : a.sc->beta;
        xa = a.sc->x_alpha;
    }
    const int t = threadIdx.x;
    if (t == 0) s_emax = 0;
    __syncthreads();

    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        const int64_t eb = e * N3;
        // ---- stage the element (raw FP64 first, to find its scale)
        int emax = 0;
        for (int q = t; q < N3; q += T) {
            double v;
            if (MODE == 1) {
                // x += alpha p of the previous iteration, then p = r + beta p
                const double pold = a.p[eb + q];
                if (xa != 0.0) a.x[eb + q] = fma(xa, pold, a.x[eb + q]);
                v = fma(beta, pold, a.r[eb + q]);
                a.p[eb + q] = v;
            } else {
                v = __ldg(a.u + eb + q);
            }
            raw[q] = v;
            const int ex = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
            emax = ex > emax ? ex : emax;
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        if ((t & 31) == 0) atomicMax(&s_emax, emax);
        __syncthreads();
        int eu = s_emax;
        eu = eu < 1 ? 1 : (eu > 2046 ? 2046 : eu);
        // u is scaled by 2^(1023-eu) so the element's max is in [1,2); w is
        // scaled back by 2^(eu-1023) and by the gxyz scale 2^(gexp-1023)
        const int sh_in = 1023 - eu;
        const int sh_out = (eu - 1023) + (a.gexp - 1023);
        for (int q = t; q < N3; q += T) U[q] = dfa::split_scaled(raw[q], sh_in);  // own entries only
        __syncthreads();

        // ---- forward: wr, ws, wt along this thread's line
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            float2 *Wd = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
            if constexpr (EO)
                line_eo<N>(U, Wd, base, stride, D.fwd);
            else
                line_plain<N, false>(U, Wd, base, stride, D);
        }
        __syncthreads();

        // ---- geometric contraction, pointwise, in place
        const float2 *g = a.g + e * 6 * N3;
        for (int q = t; q < N3; q += T) {
            const float2 wr = W0[q], ws = W1[q], wt = W2[q];
            const float2 g0 = g[q], g1 = g[N3 + q], g2 = g[2 * N3 + q];
            const float2 g3 = g[3 * N3 + q], g4 = g[4 * N3 + q], g5 = g[5 * N3 + q];
            dfa::Acc r = dfa::first(g0.x, g0.y, wr.x, wr.y);
            dfa::fma(r, g1.x, g1.y, ws.x, ws.y);
            dfa::fma(r, g2.x, g2.y, wt.x, wt.y);
            dfa::Acc s = dfa::first(g1.x, g1.y, wr.x, wr.y);
            dfa::fma(s, g3.x, g3.y, ws.x, ws.y);
            dfa::fma(s, g4.x, g4.y, wt.x, wt.y);
            dfa::Acc tt = dfa::first(g2.x, g2.y, wr.x, wr.y);
            dfa::fma(tt, g4.x, g4.y, ws.x, ws.y);
            dfa::fma(tt, g5.x, g5.y, wt.x, wt.y);
            W0[q] = dfa::norm(r);
            W1[q] = dfa::norm(s);
            W2[q] = dfa::norm(tt);
        }
        __syncthreads();

        // ---- backward: w_d(m) = sum_l dxtm1(m,l) u_d(l) = sum_l D(l,m) u_d(l)
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            const float2 *Ud = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
            float2 *Pd = task < N2 ? U : (task < 2 * N2 ? P1 : P2);
            if constexpr (EO)
                line_eo<N>(Ud, Pd, base, stride, D.bwd);
            else
                line_plain<N, true>(Ud, Pd, base, stride, D);
        }
        __syncthreads();

        // ---- w = r-partial + s-partial + t-partial, scaled back, FP64 out
        int ex = 0, ey = 0, ez = 0;
        if (MODE == 1) element_coords(e, a.m, ex, ey, ez);
        for (int q = t; q < N3; q += T) {
            const float2 s = dfa::add(dfa::add(U[q], P1[q]), P2[q]);
            double wv = dfa::join_scaled(s, sh_out);
            if (MODE == 1 && a.fuse) {
                // Dirichlet points are zeroed before dssum (their sum is
                // then +0, as mask-after-dssum gives); element-interior
                // points have multiplicity 1 and are final: <w,p> here.
                const int i = q % N, j = (q / N) % N, k = q / N2;
                if (on_box_face(i, j, k, ex, ey, ez, a.m))
                    wv = 0.0;
                else if (i > 0 && i < N - 1 && j > 0 && j < N - 1 && k > 0 && k < N - 1)
                    dot = fma(wv, a.p[eb + q], dot);
            }
            a.w[eb + q] = wv;
        }
        if (t == 0) s_emax = 0;
        __syncthreads();
    }
    if (MODE == 1 && a.fuse) {
        const double b = block_sum(dot, red);
        if (t == 0) a.partials[blockIdx.x] = b;
    }
}

// ---------------------------------------------------------------- set-up
// Largest binary exponent (biased) of |x| over an array.
__global__ void max_exponent_kernel(const double *__restrict__ x, int64_t n, int *out) {
    int emax = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int ex = (int)((__double_as_longlong(x[q]) >> 52) & 0x7ff);
        emax = ex > emax ? ex : emax;
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((threadIdx.x & 31) == 0) atomicMax(out, emax);
}

__global__ void split_scaled_kernel(const double *__restrict__ x, float2 *__restrict__ y, int64_t n,
                                    const int *eptr) {
    int ex = *eptr;
    ex = ex < 1 ? 1 : (ex > 2046 ? 2046 : ex);
    const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        y[q] = dfa::split(x[q] * sc);
}

nb_status prepare_df(nb_ctx *c) {
    const int64_t ng = (int64_t)6 * c->m.n * c->m.n * c->m.n * c->m.E;
    cudaError_t e = dev_alloc((void **)&c->d_gxyz_df, sizeof(float2) * ng);
    if (e != cudaSuccess) return cuda_fail(e, "alloc gxyz pairs");
    c->device_bytes += sizeof(float2) * ng;
    int *d_ex = nullptr;
    if ((e = dev_alloc((void **)&d_ex, sizeof(int))) != cudaSuccess) return cuda_fail(e, "alloc exponent");
    int gexp = 0;
    e = cudaMemsetAsync(d_ex, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        max_exponent_kernel<<<1024, 256, 0, c->stream>>>(c->d_gxyz, ng, d_ex);
        split_scaled_kernel<<<1024, 256, 0, c->stream>>>(c->d_gxyz, c->d_gxyz_df, ng, d_ex);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&gexp, d_ex, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_ex);
    if (e != cudaSuccess) return cuda_fail(e, "split gxyz");
    gexp = gexp < 1 ? 1 : (gexp > 2046 ? 2046 : gexp);
    c->gxyz_exp = gexp;
    c->d_eo = centro_antisymmetric(c->D_host, c->m.n);
    return NB_OK;
}

bool df_supported(int n) { return n >= 2 && n <= kMaxN; }

// Even-odd constants of M (M = D, or D^T when tr) from the FP64 matrix.
template <int N>
static void eo_consts(const double *Dm, bool tr, EoMat<N> &E) {
    constexpr int H = N / 2;
    auto M = [&](int m, int l) { return tr ? Dm[l * N + m] : Dm[m * N + l]; };
    auto put = [](double v, float &h, float &l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int m = 0; m < H; m++) {
        for (int l = 0; l < H; l++) put(0.5 * (M(m, l) + M(N - 1 - m, l)), E.ah[m * H + l], E.al[m * H + l]);
        for (int l = 0; l <= H; l++) {
            const double v = l < H ? 0.5 * (M(m, l) - M(N - 1 - m, l)) : ((N & 1) ? M(m, H) : 0.0);
            put(v, E.bh[m * (H + 1) + l], E.bl[m * (H + 1) + l]);
        }
    }
    for (int l = 0; l <= H; l++) put((N & 1) ? M(H, l) : 0.0, E.ch[l], E.cl[l]);
}

// True when D(i,l) = -D(n-1-i, n-1-l) to rounding (GLL derivative matrices).
bool centro_antisymmetric(const double *D, int n) {
    double mx = 0.0, asym = 0.0;
    for (int q = 0; q < n * n; q++) mx = fmax(mx, fabs(D[q]));
    for (int i = 0; i < n; i++)
        for (int l = 0; l < n; l++)
            asym = fmax(asym, fabs(D[i * n + l] + D[(n - 1 - i) * n + (n - 1 - l)]));
    return asym <= 1e-14 * mx;
}

template <int N, bool EO>
static nb_status launch_df_nv(nb_ctx *c, const double *u, double *w, int mode) {
    constexpr int T = ax_df_threads(N);
    const size_t smem = sizeof(float2) * 6 * N * N * N;
    static bool configured[2] = {false, false};
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    typename DfConsts<N, EO>::type D;
    if constexpr (EO) {
        eo_consts<N>(c->D_host, false, D.fwd);
        eo_consts<N>(c->D_host, true, D.bwd);
    } else {
        for (int q = 0; q < N * N; q++) {
            const float h = (float)c->D_host[q];
            D.h[q] = h;
            D.l[q] = (float)(c->D_host[q] - (double)h);
        }
    }
    AxDfArgs args{};
    args.g = c->d_gxyz_df;
    args.gexp = c->gxyz_exp;
    args.E = c->m.E;
    if (mode == 0) {
        args.u = u;
        args.w = w;
    } else {
        args.r = c->d_r;
        args.p = c->d_p;
        args.x = c->d_x;
        args.w = c->d_w;
        args.sc = c->d_sc;
        args.partials = c->d_partials;
        args.fuse = c->fused_cg ? 1 : 0;
    }
    args.m = c->m;
    auto kern = mode == 0 ? ax_df_kernel<N, 0, EO> : ax_df_kernel<N, 1, EO>;
    if (!configured[mode]) {
        NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[mode] = true;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, smem);
    if (occ < 1) occ = 1;
    const int64_t cap = (int64_t)sms * occ;
    const int grid = (int)(c->m.E < cap ? c->m.E : cap);
    if (mode == 1) c->ax_grid = grid;
    LaunchTimer tm(c, NB_K_AX);
    kern<<<grid, T, smem, c->stream>>>(args, D);
    NB_LAUNCH_CHECK("ax_df_kernel");
    return NB_OK;
}

template <int N>
static nb_status launch_df_n(nb_ctx *c, const double *u, double *w, int mode) {
    return c->d_eo ? launch_df_nv<N, true>(c, u, w, mode) : launch_df_nv<N, false>(c, u, w, mode);
}

nb_status launch_ax_df(nb_ctx *c, const double *u, double *w, int mode) {
    switch (c->m.n) {
#define NB_CASE(NN) case NN: return launch_df_n<NN>(c, u, w, mode);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
}

}  // namespace nekgb
