// Mixed-precision defect correction (iterative refinement) around an FP32
// inner CG.  The paper computes everything in FP64 (Sec. III.A); this path
// keeps the FP64 pieces that decide the answer -- the residual
// r = f - A x with the FP64-accurate operator, every dot product and norm,
// and the solution update x += d -- and runs the inner correction solve
// A d = r with FP32 u, w and gxyz in ax_e and dssum, which halves the
// operator's bytes.
//
//   x = x0
//   loop: r = f - A x (FP64);  stop if sqrt(<r,r>_c/<f,f>_c) <= tol
//         d = CG_fp32(A, r) to a relative inner residual (1e-4 by default)
//         x += d (FP64)
//
// The inner CG is the two-kernel iteration of the FP64 solver on FP32
// vectors (the FP32 head, then assemble_update): dot products accumulate
// with compensated FP32 sums into FP64 partials, and all scalars are FP64
// on the device.
#include <math.h>
#include <stdlib.h>

#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

nb_status launch_ax_f32(nb_ctx *c, const float *u, float *w, int mode);
nb_status launch_dssum_sc(nb_ctx *c, double *w, const CgScalars *sc);
nb_status launch_mask_sc(nb_ctx *c, double *w, const CgScalars *sc);
nb_status launch_ax(nb_ctx *c, const double *u, double *w);
nb_status dot_start(nb_ctx *c, const double *f);   // cg.cu: r = f - w, rho, fnorm2
nb_status launch_assemble_update32(nb_ctx *c);     // assemble.cu

constexpr int kT = 256;

static int sms32() { return device_sms(); }

__global__ void to_f32_kernel(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        y[q] = __double2float_rn(x[q]);
}

// x += (double) d
__global__ void add_f32_kernel(double *__restrict__ x, const float *__restrict__ d, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        x[q] += (double)d[q];
}

// Inner start: p = 0, x = 0, rho = <r,r>_c, fnorm2 = rho (the inner
// tolerance is relative to the inner right-hand side).
template <int N>
__global__ void __launch_bounds__(kT)
inner_start_kernel(const float *__restrict__ r, float *__restrict__ p, float *__restrict__ x, Mesh m,
                   double *partials, CgScalars *sc) {
    constexpr int N3 = N * N * N;
    dfa::Acc32 acc;   // exact products, compensated sums (FP64-class <r,r>_c)
    for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const int64_t base = e * N3;
#pragma unroll 4
        for (int q = threadIdx.x; q < N3; q += kT) {
            const int i = q % N, j = (q / N) % N, k = q / (N * N);
            const float rv = r[base + q];
            p[base + q] = 0.f;
            x[base + q] = 0.f;
            const float cw = __uint_as_float((unsigned)(127 - log2_mult(i, j, k, ex, ey, ez, m)) << 23);  // 2^-lg
            acc.add_prod(rv * cw, rv);
        }
    }
    double v[1] = {acc.value()}, tot[1];
    if (!last_block_reduce<1>(v, partials, 0, blockIdx.x, gridDim.x, gridDim.x, &sc->ticket, tot)) return;
    if (threadIdx.x != 0) return;
    sc->rho = tot[0];
    sc->rr = tot[0];
    sc->rho_old = 1.0;
    sc->fnorm2 = tot[0];
    sc->beta = 0.0;
    sc->x_alpha = 0.0;
    sc->it = 0;
    sc->status = 0;
    sc->done = (tot[0] == 0.0 || sc->maxit == 0) ? 1 : 0;
}

__global__ void inner_final_kernel(float *__restrict__ x, const float *__restrict__ p, int64_t n,
                                   const CgScalars *__restrict__ sc) {
    const float xa = (float)sc->x_alpha;
    if (xa == 0.f) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        x[q] = fmaf(xa, p[q], x[q]);
}

// ---------------------------------------------------------------- host
#define NB_DISPATCH_N32(n, CALL)                                                            \
    switch (n) {                                                                            \
        case 2: CALL(2); break; case 3: CALL(3); break; case 4: CALL(4); break;             \
        case 5: CALL(5); break; case 6: CALL(6); break; case 7: CALL(7); break;             \
        case 8: CALL(8); break; case 9: CALL(9); break; case 10: CALL(10); break;           \
        case 11: CALL(11); break; case 12: CALL(12); break; case 13: CALL(13); break;       \
        case 14: CALL(14); break; case 15: CALL(15); break; case 16: CALL(16); break;       \
        default: break;                                                                     \
    }

static int grid_e(const nb_ctx *c) {
    const int64_t cap = (int64_t)sms32() * 4;
    return (int)(c->m.E < cap ? c->m.E : cap);
}

static nb_status inner_start(nb_ctx *c) {
    LaunchTimer tm(c, NB_K_DOT);
#define CALL(NN)                                                                                    \
    inner_start_kernel<NN><<<grid_e(c), kT, 0, c->stream>>>(c->d_r32, c->d_p32, c->d_z32, c->m,    \
                                                            c->d_partials, c->d_sc)
    NB_DISPATCH_N32(c->m.n, CALL)
#undef CALL
    NB_LAUNCH_CHECK("inner_start_kernel");
    return NB_OK;
}

// One inner iteration: the FP32 head (whose last CTA forms alpha), then
// dssum fused with the residual update (assemble.cu).
static nb_status inner_iteration(nb_ctx *c) {
    nb_status s;
    if ((s = launch_ax_f32(c, nullptr, nullptr, 1)) != NB_OK) return s;
    return launch_assemble_update32(c);
}

static nb_status build_graph32(nb_ctx *c, int chunk) {
    if (c->cg_graph32 && c->cg_graph32_chunk == chunk) return NB_OK;
    if (c->cg_graph32) {
        cudaGraphExecDestroy(c->cg_graph32);
        c->cg_graph32 = nullptr;
    }
    cudaGraph_t g = nullptr;
    NB_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    nb_status s = NB_OK;
    c->capturing = true;
    c->capture_count = 0;
    for (int k = 0; k < chunk && s == NB_OK; k++) s = inner_iteration(c);
    c->capturing = false;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != NB_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->cg_graph32, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->cg_graph32_chunk = chunk;
    c->cg_graph32_kernels = c->capture_count;
    return NB_OK;
}

nb_status prepare_fp32(nb_ctx *c) {
    const int64_t ng = (int64_t)6 * c->m.n * c->m.n * c->m.n * c->m.E;
    const int64_t np = c->m.npts;
    cudaError_t e;
    if ((e = dev_alloc((void **)&c->d_gxyz32, sizeof(float) * ng)) != cudaSuccess)
        return cuda_fail(e, "alloc gxyz fp32");
    float **vecs[] = {&c->d_r32, &c->d_p32, &c->d_w32, &c->d_z32};
    for (float **v : vecs)
        if ((e = dev_alloc((void **)v, sizeof(float) * np)) != cudaSuccess)
            return cuda_fail(e, "alloc fp32 vector");
    c->device_bytes += sizeof(float) * (ng + 4 * np);
    to_f32_kernel<<<sms32() * 8, kT, 0, c->stream>>>(c->d_gxyz, c->d_gxyz32, ng);
    NB_LAUNCH_CHECK("to_f32_kernel");
    return NB_OK;
}

nb_status cg_solve_mixed(nb_ctx *c, const double *f, double *x, double tol, int maxit, int *iters,
                         double *relres) {
    nb_status s;
    if ((s = ensure_cg_workspace(c)) != NB_OK) return s;
    if (c->d_mask) return fail(NB_ERR_STATE, "the mixed-precision solve supports the box mask only");
    c->two_kernel = true;   // inner iterations: head + assemble_update
    const double inner_tol = c->mixed_inner_tol > 0.0 ? c->mixed_inner_tol : 1e-4;
    const int max_outer = c->mixed_max_outer > 0 ? c->mixed_max_outer : 50;
    const size_t bytes = sizeof(double) * c->m.npts;
    const int64_t np = c->m.npts;
    const int vgrid = grid_blocks(np, kT, sms32() * 8);
    const bool use_graph = c->stream != nullptr && !c->timing;
    NB_CUDA(cudaMemcpyAsync(c->d_x, x, bytes, cudaMemcpyDeviceToDevice, c->stream));
    int inner_total = 0, outer = 0;
    double rel = 0.0;
    bool converged = false;
    for (;;) {
        // r = f - A x in FP64 (FP64-accurate operator), rho = <r,r>_c, <f,f>_c
        CgScalars init{};
        init.tol = tol;
        init.maxit = 1;
        *c->h_sc = init;
        NB_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream));
        if ((s = launch_ax(c, c->d_x, c->d_w)) != NB_OK) return s;
        if ((s = launch_dssum_sc(c, c->d_w, nullptr)) != NB_OK) return s;
        if ((s = launch_mask_sc(c, c->d_w, nullptr)) != NB_OK) return s;
        if ((s = dot_start(c, f)) != NB_OK) return s;
        NB_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
        NB_CUDA(cudaStreamSynchronize(c->stream));
        const double rho = c->h_sc->rr, fn2 = c->h_sc->fnorm2;
        rel = fn2 > 0.0 ? sqrt(rho) / sqrt(fn2) : 0.0;
        if (rho == 0.0 || (tol > 0.0 && rel <= tol)) {
            converged = true;
            break;
        }
        if (outer >= max_outer || inner_total >= maxit) break;
        // inner FP32 CG on A d = r
        {
            LaunchTimer tm(c, NB_K_OTHER);
            to_f32_kernel<<<vgrid, kT, 0, c->stream>>>(c->d_r, c->d_r32, np);
            NB_LAUNCH_CHECK("to_f32_kernel");
        }
        CgScalars in{};
        in.tol = inner_tol;
        in.maxit = maxit - inner_total;
        *c->h_sc = in;
        NB_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream));
        if ((s = inner_start(c)) != NB_OK) return s;
        const int chunk = 16;
        int launched = 0;
        const int budget = maxit - inner_total;
        while (launched < budget) {
            if (use_graph) {
                if ((s = build_graph32(c, chunk)) != NB_OK) return s;
                NB_CUDA(cudaGraphLaunch(c->cg_graph32, c->stream));
                c->n_launched += c->cg_graph32_kernels;
                launched += chunk;
            } else {
                for (int k = 0; k < chunk && launched < budget; k++, launched++)
                    if ((s = inner_iteration(c)) != NB_OK) return s;
            }
            NB_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
            NB_CUDA(cudaStreamSynchronize(c->stream));
            if (c->h_sc->done) break;
        }
        {
            LaunchTimer tm(c, NB_K_OTHER);
            inner_final_kernel<<<vgrid, kT, 0, c->stream>>>(c->d_z32, c->d_p32, np, c->d_sc);
            add_f32_kernel<<<vgrid, kT, 0, c->stream>>>(c->d_x, c->d_z32, np);
            NB_LAUNCH_CHECK("inner_final/add");
        }
        NB_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
        NB_CUDA(cudaStreamSynchronize(c->stream));
        const int done_inner = c->h_sc->it;
        inner_total += done_inner;
        outer += 1;
        if (c->h_sc->status != 0 || done_inner == 0) break;
    }
    NB_CUDA(cudaMemcpyAsync(x, c->d_x, bytes, cudaMemcpyDeviceToDevice, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    if ((s = harvest_timing(c)) != NB_OK) return s;
    c->last_iters = inner_total;
    c->last_outer = outer;
    if (iters) *iters = inner_total;
    if (relres) *relres = rel;
    if (c->h_sc->status == (int)NB_ERR_TIMEOUT)
        return fail(NB_ERR_TIMEOUT, "a bounded device wait of the FP32 head ran out (copies drained)");
    if (c->h_sc->status == (int)NB_ERR_BREAKDOWN && !converged)
        return fail(NB_ERR_BREAKDOWN, "inner CG breakdown: <Ap,p>_c <= 0 or not finite");
    if (tol > 0.0 && !converged) return fail(NB_ERR_NOT_CONVERGED, "defect correction did not reach tol");
    return NB_OK;
}

}  // namespace nekgb
