// FP32 ax_e for the inner solve of the mixed-precision defect correction:
// Listing 1 (arXiv 2005.13425, Sec. III) with FP32 u, w and gxyz, which
// halves the operator's bytes (32 B per point instead of 64).
//
// Same line-thread layout as the double-float kernel (ax_df.cu): 3n^2
// threads own one 1-D line each; D entries are compile-time-indexed kernel
// parameters (constant-bank operands); a pointwise pass contracts with the
// six geometric factors; the transposed derivatives go to three partial
// arrays that a final pass adds.  Plain FP32 fused multiply-adds.
#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

template <int N>
struct F32Mat {
    float d[N * N];   // d[m*N + l] = D(m, l)
};

struct AxF32Args {
    const float *u;       // MODE 0 input
    float *w;             // output
    const float *r;       // MODE 1: inner residual
    float *p;             // MODE 1: inner search direction
    float *x;             // MODE 1: inner solution, receives the owed update
    const CgScalars *sc;  // MODE 1
    double *partials;     // MODE 1: one <w,p> partial per CTA (element interiors)
    Mesh m;
    const float *g;       // gxyz [E][6][n^3], FP32
    int64_t E;
};

__host__ __device__ constexpr int ax_f32_threads(int n) {
    return n <= 12 ? ((3 * n * n + 31) / 32) * 32 : ((3 * n * n + 1) / 2 + 31) / 32 * 32;
}

template <int N>
__device__ __forceinline__ int f32_line_of(int task, int &stride) {
    constexpr int N2 = N * N;
    const int d = task / N2;
    const int c = task - d * N2;
    const int a0 = c % N, a1 = c / N;
    if (d == 0) { stride = 1; return N * (a0 + N * a1); }
    if (d == 1) { stride = N; return a0 + N2 * a1; }
    stride = N2;
    return a0 + N * a1;
}

// Asynchronous global->shared copies (cp.async, no register staging): the
// element's geometric factors stream into shared memory while the forward
// derivatives are computed.  16-byte chunks when the slab is 16-byte
// aligned (n even), 4-byte otherwise.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// MODE 0: w = ax_e(u).  MODE 1: inner CG head (x += x_alpha p, p = r + beta
// p, w = ax_e(p), box faces zeroed, element-interior <w,p> per CTA).
template <int N, int MODE>
__global__ void __launch_bounds__(ax_f32_threads(N))
ax_f32_kernel(AxF32Args a, const __grid_constant__ F32Mat<N> D) {
    constexpr int N2 = N * N, N3 = N * N * N;
    constexpr int T = ax_f32_threads(N);
    extern __shared__ __align__(16) float smf[];
    float *U = smf, *W0 = smf + N3, *W1 = smf + 2 * N3, *W2 = smf + 3 * N3;
    float *P1 = smf + 4 * N3, *P2 = smf + 5 * N3;
    float *G = smf + ((6 * N3 + 3) / 4) * 4;   // 6 N3 geometric factors, 16-byte aligned
    __shared__ double red[32];
    float beta = 0.f, xa = 0.f;
    dfa::Acc32 dot;
    if (MODE == 1) {
        if (a.sc->done) return;
        beta = a.sc->it == 0 ? 0.f : (float)a.sc->beta;
        xa = (float)a.sc->x_alpha;
    }
    const int t = threadIdx.x;
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        const int64_t eb = e * N3;
        for (int q = t; q < N3; q += T) {
            float v;
            if (MODE == 1) {
                const float pold = a.p[eb + q];
                if (xa != 0.f) a.x[eb + q] = fmaf(xa, pold, a.x[eb + q]);
                v = fmaf(beta, pold, a.r[eb + q]);
                a.p[eb + q] = v;
            } else {
                v = __ldg(a.u + eb + q);
            }
            U[q] = v;
        }
        {   // prefetch this element's gxyz (consumed after the forward phase)
            const float *gsrc = a.g + e * 6 * N3;
            if ((N3 % 4) == 0) {
                for (int q = t; q < 6 * N3 / 4; q += T) cp_async16(G + 4 * q, gsrc + 4 * q);
            } else {
                for (int q = t; q < 6 * N3; q += T) cp_async4(G + q, gsrc + q);
            }
            cp_async_commit();
        }
        __syncthreads();
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = f32_line_of<N>(task, stride);
            float *Wd = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
            float x[N];
#pragma unroll
            for (int l = 0; l < N; l++) x[l] = U[base + l * stride];
#pragma unroll
            for (int m = 0; m < N; m++) {
                float acc = D.d[m * N] * x[0];
#pragma unroll
                for (int l = 1; l < N; l++) acc = fmaf(D.d[m * N + l], x[l], acc);
                Wd[base + m * stride] = acc;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int q = t; q < N3; q += T) {
            const float wr = W0[q], ws = W1[q], wt = W2[q];
            const float g0 = G[q], g1 = G[N3 + q], g2 = G[2 * N3 + q];
            const float g3 = G[3 * N3 + q], g4 = G[4 * N3 + q], g5 = G[5 * N3 + q];
            W0[q] = fmaf(g0, wr, fmaf(g1, ws, g2 * wt));
            W1[q] = fmaf(g1, wr, fmaf(g3, ws, g4 * wt));
            W2[q] = fmaf(g2, wr, fmaf(g4, ws, g5 * wt));
        }
        __syncthreads();
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = f32_line_of<N>(task, stride);
            const float *Ud = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
            float *Pd = task < N2 ? U : (task < 2 * N2 ? P1 : P2);
            float x[N];
#pragma unroll
            for (int l = 0; l < N; l++) x[l] = Ud[base + l * stride];
#pragma unroll
            for (int m = 0; m < N; m++) {
                float acc = D.d[m] * x[0];
#pragma unroll
                for (int l = 1; l < N; l++) acc = fmaf(D.d[l * N + m], x[l], acc);
                Pd[base + m * stride] = acc;
            }
        }
        __syncthreads();
        int ex = 0, ey = 0, ez = 0;
        if (MODE == 1) element_coords(e, a.m, ex, ey, ez);
        for (int q = t; q < N3; q += T) {
            float wv = U[q] + P1[q] + P2[q];
            if (MODE == 1) {
                const int i = q % N, j = (q / N) % N, k = q / N2;
                if (on_box_face(i, j, k, ex, ey, ez, a.m))
                    wv = 0.f;
                else if (i > 0 && i < N - 1 && j > 0 && j < N - 1 && k > 0 && k < N - 1)
                    dot.add_prod(wv, a.p[eb + q]);
            }
            a.w[eb + q] = wv;
        }
        __syncthreads();
    }
    if (MODE == 1) {
        const double b = block_sum(dot.value(), red);
        if (t == 0) a.partials[blockIdx.x] = b;
    }
}

template <int N>
static nb_status launch_f32_n(nb_ctx *c, const float *u, float *w, int mode) {
    constexpr int T = ax_f32_threads(N);
    const size_t smem = sizeof(float) * (((6 * N * N * N + 3) / 4) * 4 + 6 * N * N * N);
    static bool configured[2] = {false, false};
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    F32Mat<N> D;
    for (int q = 0; q < N * N; q++) D.d[q] = (float)c->D_host[q];
    AxF32Args args{};
    args.g = c->d_gxyz32;
    args.E = c->m.E;
    args.m = c->m;
    if (mode == 0) {
        args.u = u;
        args.w = w;
    } else {
        args.r = c->d_r32;
        args.p = c->d_p32;
        args.x = c->d_z32;
        args.w = c->d_w32;
        args.sc = c->d_sc;
        args.partials = c->d_partials;
    }
    auto kern = mode == 0 ? ax_f32_kernel<N, 0> : ax_f32_kernel<N, 1>;
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
    NB_LAUNCH_CHECK("ax_f32_kernel");
    return NB_OK;
}

nb_status launch_ax_f32(nb_ctx *c, const float *u, float *w, int mode) {
    switch (c->m.n) {
#define NB_CASE(NN) case NN: return launch_f32_n<NN>(c, u, w, mode);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
}

}  // namespace nekgb
