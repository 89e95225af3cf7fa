// FP32 ax_e for the inner solve of the mixed-precision defect correction:
// Listing 1 (arXiv 2005.13425, Sec. III) with FP32 u, w and gxyz, which
// halves the operator's bytes (32 B per point instead of 64).
//
// Same line-thread layout as the double-float kernel (ax_df.cu): 3n^2
// threads own one 1-D line each; D entries are compile-time-indexed kernel
// parameters (constant-bank operands); a pointwise pass contracts with the
// six geometric factors; the transposed derivatives go to three partial
// arrays that a final pass adds.  Plain FP32 fused multiply-adds.
#include "ax_f32_core.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

struct AxF32Args {
    const float *u;       // MODE 0 input
    float *w;             // output
    const float *r;       // MODE 1: inner residual
    float *p;             // MODE 1: inner search direction
    float *x;             // MODE 1: inner solution, receives the owed update
    CgScalars *sc;        // MODE 1
    double *partials;     // MODE 1: one <w,p> partial per CTA (local products)
    int finalize;         // MODE 1: the last CTA reduces <w,p>_c and forms alpha
    Mesh m;
    const float *g;       // gxyz [E][6][n^3], FP32
    int64_t E;
    uint64_t unarmed_wait_ns;  // staged kernel, tests only: 0, or the limit of a first wait on a
                               // barrier nothing arrives on (exercises the timeout path)
};

// MODE 0: w = ax_e(u).  MODE 1: inner CG head (x += x_alpha p, p = r + beta
// p, w = ax_e(p), box faces zeroed, the local products w p per CTA; with
// finalize the last CTA forms alpha).
template <int N, int MODE>
__global__ void __launch_bounds__(ax_f32_threads(N))
ax_f32_kernel(AxF32Args a, const __grid_constant__ F32Mat<N> D) {
    constexpr int N3 = N * N * N;
    constexpr int T = ax_f32_threads(N);
    extern __shared__ __align__(16) float smf[];
    __shared__ double red[32];
    float beta = 0.f, xa = 0.f;
    dfa::Acc32 dot;
    if (MODE == 1) {
        if (a.sc->done) return;
        beta = a.sc->it == 0 ? 0.f : (float)a.sc->beta;
        xa = (float)a.sc->x_alpha;
    }
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        const int64_t eb = e * N3;
        F32ElemIO io;
        io.u = MODE == 0 ? a.u + eb : nullptr;
        io.r = MODE == 1 ? a.r + eb : nullptr;
        io.p = MODE == 1 ? a.p + eb : nullptr;
        io.x = MODE == 1 ? a.x + eb : nullptr;
        io.w = a.w + eb;
        io.g = a.g + e * 6 * N3;
        int ex = 0, ey = 0, ez = 0;
        if (MODE == 1) element_coords(e, a.m, ex, ey, ez);
        f32_element<N, MODE, T>(io, beta, xa, ex, ey, ez, a.m, D, smf, dot);
    }
    if (MODE == 1) {
        if (a.finalize) {
            double v[1] = {dot.value()}, tot[1];
            if (last_block_reduce<1>(v, a.partials, 0, blockIdx.x, gridDim.x, gridDim.x, &a.sc->ticket, tot) &&
                threadIdx.x == 0)
                finalize_alpha(a.sc, tot[0]);
        } else {
            const double b = block_sum(dot.value(), red);
            if (threadIdx.x == 0) a.partials[blockIdx.x] = b;
        }
    }
}

// The same operator with bulk-copy staging two elements deep (see
// f32_element_staged): thread 0 arms the next element's barrier and issues
// its copies, every thread waits (bounded) for the current one.  A copy
// that does not complete within ~1 s ends the kernel with NB_ERR_TIMEOUT in
// the scalar block (err), after draining the copies in flight.  With
// unarmed_wait_ns (a context set up with NEKGB_TEST_UNARMED_WAIT_NS, for
// tests) each CTA's first wait is made on a barrier that nothing arrives on,
// with that limit: it runs out, and the same drain-and-report path runs.
template <int N, int MODE>
__global__ void __launch_bounds__(ax_f32_threads(N), f32_staged_min_blocks<N>())
ax_f32_staged_kernel(AxF32Args a, CgScalars *err, const __grid_constant__ F32Mat<N> D) {
    constexpr int N3 = N * N * N;
    constexpr int T = ax_f32_threads(N);
    constexpr int STAGE = f32_stage_floats<N, MODE>();
    extern __shared__ __align__(16) float smf[];
    __shared__ double red[32];
    __shared__ __align__(8) uint64_t bars[3];   // bars[2] is never armed (unarmed_wait_ns)
    float beta = 0.f, xa = 0.f;
    dfa::Acc32 dot;
    if (MODE == 1) {
        if (a.sc->done) return;
        beta = a.sc->it == 0 ? 0.f : (float)a.sc->beta;
        xa = (float)a.sc->x_alpha;
    }
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool with_x = MODE == 1 && xa != 0.f;
    const unsigned bytes = 4u * (MODE == 1 ? (with_x ? 3 : 2) : 1) * N3;
    // x is read once per iteration: evict it first, so p and w stay in L2
    // for the update kernel (the geometric factors are streamed into
    // registers with evict-first loads by the element body)
    const uint64_t stream_pol = t == 0 ? l2_evict_first_policy() : 0ull;
    auto issue = [&](int64_t e, int s) {   // thread 0
        float *st = smf + s * STAGE;
        mbar_expect_tx(&bars[s], bytes);
        if (MODE == 1) {
            bulk_g2s(st, a.r + e * N3, 4u * N3, &bars[s]);
            bulk_g2s(st + N3, a.p + e * N3, 4u * N3, &bars[s]);
            if (with_x) bulk_g2s_hint(st + 2 * N3, a.x + e * N3, 4u * N3, &bars[s], stream_pol);
        } else {
            bulk_g2s(st, a.u + e * N3, 4u * N3, &bars[s]);
        }
    };
    int issued[2] = {0, 0}, waited[2] = {0, 0};
    unsigned pf[f32_points_per_thread<N, T>()];
    f32_point_masks<N, T>(pf);
    int64_t e = blockIdx.x;
    if (t == 0 && e < a.E) issue(e, 0);
    issued[0] = e < a.E ? 1 : 0;
    bool ok = true;
    float gv[f32_points_per_thread<N, T>()][6];
    if (e < a.E) f32_load_factors<N, T>(a.g + e * 6 * N3, gv);
    for (int i = 0; e < a.E; e += gridDim.x, i++) {
        const int s = i & 1;
        const int64_t en = e + gridDim.x;
        if (en < a.E) {
            if (t == 0) issue(en, s ^ 1);
            issued[s ^ 1]++;
        }
        const bool unarmed = a.unarmed_wait_ns != 0 && i == 0;
        ok = __syncthreads_and(unarmed ? mbar_wait(&bars[2], 0, a.unarmed_wait_ns)
                                       : mbar_wait(&bars[s], waited[s] & 1)) != 0;
        if (!ok) break;
        waited[s]++;
        F32StagedOut o;
        o.p = MODE == 1 ? a.p + e * N3 : nullptr;
        o.x = MODE == 1 ? a.x + e * N3 : nullptr;
        o.w = a.w + e * N3;
        int ex = 0, ey = 0, ez = 0;
        if (MODE == 1) element_coords(e, a.m, ex, ey, ez);
        f32_element_staged<N, MODE, T>(smf + s * STAGE, smf + 2 * STAGE, gv, en < a.E ? a.g + en * 6 * N3 : nullptr,
                                       o, beta, xa, ex, ey, ez, a.m, D, dot, pf);
    }
    if (!ok) {   // drain the copies in flight before leaving, then report
        if (t == 0) {
            for (int s = 0; s < 2; s++)
                if (issued[s] > waited[s]) mbar_wait(&bars[s], waited[s] & 1);
            if (err) {
                err->status = (int)NB_ERR_TIMEOUT;
                err->done = 1;
            }
        }
        __syncthreads();
    }
    if (MODE == 1) {
        if (a.finalize) {
            double v[1] = {dot.value()}, tot[1];
            if (last_block_reduce<1>(v, a.partials, 0, blockIdx.x, gridDim.x, gridDim.x, &a.sc->ticket, tot) &&
                threadIdx.x == 0)
                finalize_alpha(a.sc, tot[0]);
        } else {
            const double b = block_sum(dot.value(), red);
            if (threadIdx.x == 0) a.partials[blockIdx.x] = b;
        }
    }
}

template <int N>
static nb_status launch_f32_n(nb_ctx *c, const float *u, float *w, int mode) {
    constexpr int T = ax_f32_threads(N);
    const size_t smem = sizeof(float) * f32_smem_floats(N);
    int occ = 0;
    const int sms = device_sms();
    F32Mat<N> D;
    for (int q = 0; q < N * N; q++) D.d[q] = (float)c->D_host[q];
    AxF32Args args{};
    args.g = c->d_gxyz32;
    args.E = c->m.E;
    args.m = c->m;
    args.unarmed_wait_ns = c->test_unarmed_wait_ns;
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
        args.finalize = c->two_kernel ? 1 : 0;
    }
    if constexpr (f32_staged_ok<N>()) {
        if (!c->f32_plain) {
            auto kern = mode == 0 ? ax_f32_staged_kernel<N, 0> : ax_f32_staged_kernel<N, 1>;
            const size_t ssm = sizeof(float) * (mode == 0 ? f32_staged_smem_floats<N, 0>()
                                                          : f32_staged_smem_floats<N, 1>());
            {
                const nb_status s = set_smem(kern, ssm);
                if (s != NB_OK) return s;
            }
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, ssm);
            if (occ < 1) occ = 1;
            const int64_t cap = (int64_t)sms * occ;
            const int grid = (int)(c->m.E < cap ? c->m.E : cap);
            if (mode == 1) c->ax_grid = grid;
            LaunchTimer tm(c, NB_K_AX);
            kern<<<grid, T, ssm, c->stream>>>(args, c->d_sc, D);
            NB_LAUNCH_CHECK("ax_f32_staged_kernel");
            return NB_OK;
        }
    }
    auto kern = mode == 0 ? ax_f32_kernel<N, 0> : ax_f32_kernel<N, 1>;
    {
        const nb_status s = set_smem(kern, smem);
        if (s != NB_OK) return s;
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
