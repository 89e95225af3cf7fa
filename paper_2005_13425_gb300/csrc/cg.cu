// Unpreconditioned conjugate gradient for Ax = f on the device (arXiv
// 2005.13425 Sec. III: Nekbone solves the SEM Poisson system with CG;
// Sec. V: 100 fixed iterations; Sec. VII: no preconditioner), plus the
// deterministic weighted inner product <a,b>_c = sum a*b/multiplicity.
//
// Every scalar of the iteration (rho, alpha, beta, <w,p>_c) lives on the
// device and reductions are deterministic (reduce.cuh).  With the box mask
// and no preconditioner one iteration is two kernels:
//   1. ax_e head: x += alpha_prev p (the x update owed by the previous
//      iteration), p = r + beta p, w = ax_e(p), w := 0 on box faces, and
//      <w,p>_c as the sum of the local products w p (p is continuous, so
//      sum_g (sum_copies w) p_g equals the sum over local points); its last
//      CTA forms alpha = rho/<w,p>_c;
//   2. assemble_update (assemble.cu): dssum fused with r -= alpha w and
//      <r,r>_c; its last CTA forms rho, beta and the convergence decision.
// With the Jacobi preconditioner the dssum (forming alpha) and the update
// (with <r,z>_c) are separate kernels.  The last owed x update runs once
// after the loop.  With a caller-supplied mask array the mask may select
// any point, so the iteration falls back to separate dssum, mask and
// <w,p>_c kernels.  Chunks of iterations are captured as CUDA graphs; every
// kernel returns at once when `done` is set.
#include <math.h>

#include <mutex>

#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

nb_status launch_ax_fp64(nb_ctx *c, const double *u, double *w, int mode);
nb_status launch_ax_df(nb_ctx *c, const double *u, double *w, int mode);
bool df_supported(int n);
nb_status launch_dssum_sc(nb_ctx *c, double *w, const CgScalars *sc);
nb_status launch_dssum_cg(nb_ctx *c);
nb_status launch_mask_sc(nb_ctx *c, double *w, const CgScalars *sc);
nb_status launch_assemble_update(nb_ctx *c);
int dssum_grid(const nb_ctx *c);

constexpr int kRedThreads = 256;
constexpr int kMaxRedGrid = 16384;   // partial slots reserved per reduction

static int sms() { return device_sms(); }

// Four CTAs per SM, each striding over many elements: every CTA ends with
// one block reduction (~1.5k FP64 adds), so few, long-lived CTAs keep that
// cost far below the per-point work on GB300's narrow FP64 pipe.
static int red_grid(const nb_ctx *c) {
    const int64_t cap = (int64_t)sms() * 4;
    return (int)(c->m.E < cap ? c->m.E : cap);
}

// The update kernel: six CTAs per SM (its register bound), one wave.
static int update_grid(const nb_ctx *c) {
    const int64_t cap = (int64_t)sms() * 6;
    return (int)(c->m.E < cap ? c->m.E : cap);
}

// MODE 0: *out = <a,b>_c.
// MODE 1 (unfused solver step): pap = <w,p>_c, alpha = rho/pap.
// MODE 2 (solver start): r = f - w, p = 0, rho = <r,z>_c (z = minv r or r),
//   rr = <r,r>_c, fnorm2 = <f,f>_c.
template <int N, int MODE>
__global__ void __launch_bounds__(kRedThreads)
dot_kernel(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ rr,
           double *__restrict__ pp, Mesh m, double *partials, CgScalars *sc, double *out,
           double *hist, const double *__restrict__ minv) {
    constexpr int N3 = N * N * N;
    if (MODE == 1 && sc->done) return;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const int64_t base = e * N3;
#pragma unroll 4
        for (int p = threadIdx.x; p < N3; p += kRedThreads) {
            const int i = p % N, j = (p / N) % N, k = p / (N * N);
            const double cw = inv_mult(i, j, k, ex, ey, ez, m);
            if (MODE == 2) {
                const double f = a[base + p];
                const double r = f - b[base + p];
                rr[base + p] = r;
                pp[base + p] = 0.0;
                const int lg = log2_mult(i, j, k, ex, ey, ez, m);
                acc0 = fma(scale_down_pow2(r, lg), r, acc0);
                acc1 = fma(scale_down_pow2(f, lg), f, acc1);
                if (minv) acc2 = fma(scale_down_pow2(r * minv[base + p], lg), r, acc2);
            } else {
                acc0 = fma(a[base + p] * cw, b[base + p], acc0);
            }
        }
    }
    if (MODE == 2) {
        double v[3] = {acc0, acc1, acc2}, tot[3];
        if (!last_block_reduce<3>(v, partials, gridDim.x, blockIdx.x, gridDim.x, gridDim.x,
                                  &sc->ticket, tot))
            return;
        if (threadIdx.x != 0) return;
        sc->rr = tot[0];
        sc->rho = minv ? tot[2] : tot[0];
        sc->rho_old = 1.0;
        sc->fnorm2 = tot[1];
        sc->beta = 0.0;
        sc->x_alpha = 0.0;
        sc->it = 0;
        sc->status = 0;
        if (hist) hist[0] = tot[0];
        const bool conv = sc->tol > 0.0 && sqrt(tot[0]) / sqrt(tot[1]) <= sc->tol;
        sc->done = (sc->rho == 0.0 || conv || sc->maxit == 0) ? 1 : 0;
        return;
    }
    double v[1] = {acc0}, tot[1];
    if (!last_block_reduce<1>(v, partials, 0, blockIdx.x, gridDim.x, gridDim.x, &sc->ticket, tot))
        return;
    if (threadIdx.x != 0) return;
    if (MODE == 0) {
        *out = tot[0];
    } else {
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

// Body of the update: r -= alpha w over this CTA's elements, accumulating
// <r,r>_c and, with PRE, <r, minv r>_c (shared nodes weighted 1/multiplicity).
template <int N, bool PRE>
__device__ __forceinline__ void update_body(double *__restrict__ r, const double *__restrict__ w, const Mesh &m,
                                            double alpha, const double *__restrict__ minv, double &acc,
                                            double &accz, int sh) {
    constexpr int N3 = N * N * N;
    constexpr int K = (N3 + kRedThreads - 1) / kRedThreads;   // points per thread per element
    dfa::SqAcc32 sq;
    unsigned pf[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int q = threadIdx.x + k * kRedThreads;
        pf[k] = q < N3 ? point_faces<N>(q) : 0u;
    }
    for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const unsigned sf = shared_faces(ex, ey, ez, m);
        const int64_t base = e * N3;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int q = threadIdx.x + k * kRedThreads;
            if (K * kRedThreads != N3 && q >= N3) break;
            const double rn = fma(-alpha, __ldcs(w + base + q), r[base + q]);
            r[base + q] = rn;
            const int lg = __popc(pf[k] & sf);
            if (PRE) {
                acc = fma(scale_down_pow2(rn, lg), rn, acc);
                accz = fma(scale_down_pow2(rn * minv[base + q], lg), rn, accz);
            } else {
                // <r,r>_c on the FP32 pipes: r 2^sh split into a pair with
                // integer operations, squares accumulated compensated
                const float2 v = dfa::split_scaled<true>(rn, sh);
                sq.add_sq(v.x, v.y, __uint_as_float((127u - (unsigned)lg) << 23));
            }
        }
    }
    if (!PRE) acc = sq.value() * __longlong_as_double((long long)(1023 - 2 * sh) << 52);
}

// r -= alpha w, rr = <r,r>_c, rho = <r,z>_c (z = minv r with Jacobi, else
// rho = rr), beta = rho/rho_old, convergence decision on rr.  PRE selects
// the Jacobi form at compile time so the plain kernel carries none of it.
template <int N, bool PRE>
__global__ void __launch_bounds__(kRedThreads, 6)
update_kernel(double *__restrict__ r, const double *__restrict__ w, Mesh m, double *partials,
              CgScalars *sc, double *hist, const double *__restrict__ minv) {
    if (sc->done) return;
    const double alpha = sc->alpha;
    double acc = 0.0, accz = 0.0, rr, rho;
    // scale 2^sh with (r 2^sh)^2 of order one: from the previous <r,r>_c
    // (the residual changes by modest factors per iteration; the FP32
    // range leaves 2^+-60 of room either way)
    const int erb = (int)((__double_as_longlong(sc->rr) >> 52) & 0x7ff);
    const int sh = erb == 0 ? 0 : -((erb - 1023) >> 1);
    update_body<N, PRE>(r, w, m, alpha, minv, acc, accz, sh);
    if (PRE) {
        double v[2] = {acc, accz}, tot[2];
        if (!last_block_reduce<2>(v, partials, gridDim.x, blockIdx.x, gridDim.x, gridDim.x, &sc->ticket, tot))
            return;
        rr = tot[0];
        rho = tot[1];
    } else {
        double v[1] = {acc}, tot[1];
        if (!last_block_reduce<1>(v, partials, 0, blockIdx.x, gridDim.x, gridDim.x, &sc->ticket, tot))
            return;
        rr = tot[0];
        rho = rr;
    }
    if (threadIdx.x != 0) return;
    sc->rr = rr;
    sc->rho_old = sc->rho;
    sc->rho = rho;
    sc->beta = rho / sc->rho_old;
    const int it = sc->it + 1;
    sc->it = it;
    hist[it] = rr;
    const bool conv = sc->tol > 0.0 && sqrt(rr) / sqrt(sc->fnorm2) <= sc->tol;
    if (rho == 0.0 || conv || it >= sc->maxit) sc->done = 1;
}

// The x update owed by the last iteration: x += x_alpha p.
__global__ void final_x_kernel(double *__restrict__ x, const double *__restrict__ p, int64_t n,
                               const CgScalars *__restrict__ sc) {
    const double xa = sc->x_alpha;
    if (xa == 0.0) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        x[q] = fma(xa, p[q], x[q]);
}

// ---------------------------------------------------------------- host side
#define NB_DISPATCH_N(n, CALL)                                                              \
    switch (n) {                                                                            \
        case 2: CALL(2); break; case 3: CALL(3); break; case 4: CALL(4); break;             \
        case 5: CALL(5); break; case 6: CALL(6); break; case 7: CALL(7); break;             \
        case 8: CALL(8); break; case 9: CALL(9); break; case 10: CALL(10); break;           \
        case 11: CALL(11); break; case 12: CALL(12); break; case 13: CALL(13); break;       \
        case 14: CALL(14); break; case 15: CALL(15); break; case 16: CALL(16); break;       \
        default: break;                                                                     \
    }

template <int N>
static void dot_launch(nb_ctx *c, int mode, const double *a, const double *b, double *out) {
    const int grid = red_grid(c);
    if (mode == 0)
        dot_kernel<N, 0><<<grid, kRedThreads, 0, c->stream>>>(a, b, nullptr, nullptr, c->m, c->d_partials,
                                                             c->d_sc, out, nullptr, nullptr);
    else if (mode == 1)
        dot_kernel<N, 1><<<grid, kRedThreads, 0, c->stream>>>(c->d_w, c->d_p, nullptr, nullptr, c->m,
                                                             c->d_partials, c->d_sc, nullptr, nullptr,
                                                             nullptr);
    else
        dot_kernel<N, 2><<<grid, kRedThreads, 0, c->stream>>>(a, b, c->d_r, c->d_p, c->m, c->d_partials,
                                                             c->d_sc, nullptr,
                                                             c->prec == NB_MIXED ? nullptr : c->d_hist,
                                                             c->prec == NB_MIXED ? nullptr : c->d_minv);
}

template <int N>
static void update_launch(nb_ctx *c) {
    if (c->d_minv)
        update_kernel<N, true><<<update_grid(c), kRedThreads, 0, c->stream>>>(c->d_r, c->d_w, c->m, c->d_partials,
                                                                          c->d_sc, c->d_hist, c->d_minv);
    else
        update_kernel<N, false><<<update_grid(c), kRedThreads, 0, c->stream>>>(c->d_r, c->d_w, c->m,
                                                                           c->d_partials, c->d_sc, c->d_hist,
                                                                           nullptr);
}

static nb_status launch_dot(nb_ctx *c, int mode, const double *a, const double *b, double *out) {
    LaunchTimer tm(c, NB_K_DOT);
#define CALL(NN) dot_launch<NN>(c, mode, a, b, out)
    NB_DISPATCH_N(c->m.n, CALL)
#undef CALL
    NB_LAUNCH_CHECK("dot_kernel");
    return NB_OK;
}

static nb_status launch_update(nb_ctx *c) {
    LaunchTimer tm(c, NB_K_UPDATE);
#define CALL(NN) update_launch<NN>(c)
    NB_DISPATCH_N(c->m.n, CALL)
#undef CALL
    NB_LAUNCH_CHECK("update_kernel");
    return NB_OK;
}

static bool use_df(const nb_ctx *c) {
    return (c->ax_variant == 0 || c->ax_variant == 2) && c->d_gxyz_df && df_supported(c->m.n);
}

nb_status launch_ax(nb_ctx *c, const double *u, double *w) {
    return use_df(c) ? launch_ax_df(c, u, w, 0) : launch_ax_fp64(c, u, w, 0);
}

nb_status launch_ax_cg(nb_ctx *c) {
    return use_df(c) ? launch_ax_df(c, nullptr, nullptr, 1) : launch_ax_fp64(c, nullptr, nullptr, 1);
}

nb_status ensure_cg_workspace(nb_ctx *c) {
    if (c->d_sc) return NB_OK;
    const size_t bytes = sizeof(double) * c->m.npts;
    cudaError_t e;
    double **vecs[] = {&c->d_r, &c->d_p, &c->d_w, &c->d_x};
    for (double **v : vecs) {
        if ((e = dev_alloc((void **)v, bytes)) != cudaSuccess) return cuda_fail(e, "alloc CG vector");
        c->device_bytes += bytes;
    }
    // slots: up to 2 values x (ax_e CTAs + dssum CTAs, or a reduction grid)
    c->partial_cap = 2 * (2 * kMaxRedGrid) + 16;
    if ((e = dev_alloc((void **)&c->d_partials, sizeof(double) * c->partial_cap)) != cudaSuccess)
        return cuda_fail(e, "alloc partials");
    c->device_bytes += sizeof(double) * c->partial_cap;
    if ((e = dev_alloc((void **)&c->d_sc, sizeof(CgScalars))) != cudaSuccess)
        return cuda_fail(e, "alloc scalars");
    if ((e = cudaMallocHost((void **)&c->h_sc, sizeof(CgScalars))) != cudaSuccess)
        return cuda_fail(e, "alloc pinned scalars");
    NB_CUDA(cudaMemsetAsync(c->d_sc, 0, sizeof(CgScalars), c->stream));
    return NB_OK;
}

static nb_status ensure_hist(nb_ctx *c, int maxit) {
    if (c->d_hist && c->hist_cap >= maxit + 1) return NB_OK;
    if (c->d_hist) {
        NB_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->d_hist);
        c->d_hist = nullptr;
        if (c->cg_graph) {   // the captured iteration writes the old history buffer
            cudaGraphExecDestroy(c->cg_graph);
            c->cg_graph = nullptr;
        }
    }
    int cap = maxit + 1 < 1024 ? 1024 : maxit + 1;
    cudaError_t e = dev_alloc((void **)&c->d_hist, sizeof(double) * cap);
    if (e != cudaSuccess) return cuda_fail(e, "alloc history");
    c->hist_cap = cap;
    return NB_OK;
}

// Solver start: r = f - w, p = 0, rho = <r,r>_c, <f,f>_c (used by the
// mixed-precision outer loop; needs no history buffer).
nb_status dot_start(nb_ctx *c, const double *f) { return launch_dot(c, 2, f, c->d_w, nullptr); }

nb_status dot_c(nb_ctx *c, const double *a, const double *b, double *out_host) {
    nb_status s = ensure_cg_workspace(c);
    if (s != NB_OK) return s;
    double *d_out = c->d_partials + c->partial_cap - 1;
    if ((s = launch_dot(c, 0, a, b, d_out)) != NB_OK) return s;
    NB_CUDA(cudaMemcpyAsync(out_host, d_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    return harvest_timing(c);
}

// One CG iteration; every kernel returns at once when done is set.
static nb_status enqueue_iteration(nb_ctx *c) {
    nb_status s;
    if ((s = launch_ax_cg(c)) != NB_OK) return s;
    if (c->two_kernel) return launch_assemble_update(c);
    if (c->fused_cg) {
        if ((s = launch_dssum_cg(c)) != NB_OK) return s;
    } else {
        if ((s = launch_dssum_sc(c, c->d_w, c->d_sc)) != NB_OK) return s;
        if ((s = launch_mask_sc(c, c->d_w, c->d_sc)) != NB_OK) return s;
        if ((s = launch_dot(c, 1, nullptr, nullptr, nullptr)) != NB_OK) return s;
    }
    return launch_update(c);
}

static nb_status build_graph(nb_ctx *c, int chunk) {
    if (c->cg_graph && c->cg_graph_chunk == chunk && c->cg_graph_two == c->two_kernel) return NB_OK;
    if (c->cg_graph) {
        cudaGraphExecDestroy(c->cg_graph);
        c->cg_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    NB_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    nb_status s = NB_OK;
    c->capturing = true;
    c->capture_count = 0;
    for (int k = 0; k < chunk && s == NB_OK; k++) s = enqueue_iteration(c);
    c->capturing = false;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != NB_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->cg_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->cg_graph_chunk = chunk;
    c->cg_graph_two = c->two_kernel;
    c->cg_graph_kernels = c->capture_count;
    return NB_OK;
}

nb_status cg_solve_fp64(nb_ctx *c, const double *f, double *x, double tol, int maxit, int *iters,
                        double *relres) {
    nb_status s;
    if ((s = ensure_cg_workspace(c)) != NB_OK) return s;
    if ((s = ensure_hist(c, maxit)) != NB_OK) return s;
    c->fused_cg = c->d_mask == nullptr;
    c->two_kernel = c->fused_cg && !c->d_minv && use_df(c);
    const size_t bytes = sizeof(double) * c->m.npts;
    CgScalars init{};
    init.tol = tol;
    init.maxit = maxit;
    *c->h_sc = init;
    NB_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream));
    // x_int = x0; w = A x0; r = f - w; p = 0; rho = <r,r>_c; <f,f>_c
    NB_CUDA(cudaMemcpyAsync(c->d_x, x, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if ((s = launch_ax(c, c->d_x, c->d_w)) != NB_OK) return s;
    if ((s = launch_dssum_sc(c, c->d_w, nullptr)) != NB_OK) return s;
    if ((s = launch_mask_sc(c, c->d_w, nullptr)) != NB_OK) return s;
    if ((s = launch_dot(c, 2, f, c->d_w, nullptr)) != NB_OK) return s;

    // Stream capture needs a non-default stream; event timing needs plain
    // launches.  Sampled timing (timing = 2) runs the first iteration of
    // every chunk as plain, event-timed launches and the rest as a graph.
    const bool sampled = c->timing == 2;
    const bool use_graph = c->stream != nullptr && (!c->timing || sampled);
    const int chunk = 16;
    int launched = 0;
    while (launched < maxit) {
        if (use_graph) {
            if (sampled) {
                if ((s = enqueue_iteration(c)) != NB_OK) return s;
                launched += 1;
            }
            const int g = sampled ? chunk - 1 : chunk;
            if ((s = build_graph(c, g)) != NB_OK) return s;
            NB_CUDA(cudaGraphLaunch(c->cg_graph, c->stream));
            c->n_launched += c->cg_graph_kernels;
            launched += g;
        } else {
            for (int k = 0; k < chunk && launched < maxit; k++, launched++)
                if ((s = enqueue_iteration(c)) != NB_OK) return s;
        }
        if (tol > 0.0 && launched < maxit) {
            NB_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
            NB_CUDA(cudaStreamSynchronize(c->stream));
            if (c->h_sc->done) break;
        }
    }
    {
        LaunchTimer tm(c, NB_K_OTHER);
        const int grid = grid_blocks(c->m.npts, 256, sms() * 8);
        final_x_kernel<<<grid, 256, 0, c->stream>>>(c->d_x, c->d_p, c->m.npts, c->d_sc);
        NB_LAUNCH_CHECK("final_x_kernel");
    }
    NB_CUDA(cudaMemcpyAsync(x, c->d_x, bytes, cudaMemcpyDeviceToDevice, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    if ((s = harvest_timing(c)) != NB_OK) return s;
    const CgScalars &h = *c->h_sc;
    c->last_iters = h.it;
    if (iters) *iters = h.it;
    const double rel = h.fnorm2 > 0.0 ? sqrt(h.rr) / sqrt(h.fnorm2) : 0.0;
    if (relres) *relres = rel;
    if (h.status == (int)NB_ERR_BREAKDOWN && h.fault == kFaultExactSumRange)
        return fail(NB_ERR_BREAKDOWN, "the exact <w,p>_c sum left its range (its scale comes from the <p,p>_c recursion)");
    if (h.status == (int)NB_ERR_BREAKDOWN) return fail(NB_ERR_BREAKDOWN, "CG breakdown: <Ap,p>_c <= 0 or not finite");
    if (tol > 0.0 && !(rel <= tol) && h.rr != 0.0)
        return fail(NB_ERR_NOT_CONVERGED, "CG did not reach the tolerance within maxit");
    return NB_OK;
}

// ---------------------------------------------------------------- allocation-free dot
// Some callers cannot call cudaMalloc: code running under a memory manager
// that already owns the device memory (a framework's caching allocator, an
// application that reserves the GPU up front), and code that must not block
// (cudaMalloc and cudaFree may synchronise the device).  For them the weighted
// dot product runs the same reduction kernel with its scratch -- one
// partial sum per element plus the last-CTA ticket -- in a file-scope
// device array instead of a context's allocation.  Every GPU that loads the
// library holds this array (about 256 KB) until the process exits.
constexpr int kNoAllocMaxElements = 32768;

struct NoAllocScratch {
    double partials[kNoAllocMaxElements];
    CgScalars sc;   // only the ticket is used
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static std::mutex g_noalloc_mu;
static NoAllocScratch *g_noalloc_ptr[256];

// Device address of the scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device address).
static nb_status noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(NB_ERR_STATE, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(allocation-free scratch)");
        g_noalloc_ptr[dev] = (NoAllocScratch *)p;
    }
    *out = g_noalloc_ptr[dev];
    return NB_OK;
}

nb_status dot_c_noalloc(const Mesh &m, const double *a, const double *b, double *out,
                        cudaStream_t stream) {
    if (m.E > kNoAllocMaxElements)
        return fail(NB_ERR_ARG, "the allocation-free dot product supports at most 32768 elements");
    NoAllocScratch *s = nullptr;
    nb_status st = noalloc_scratch(&s);
    if (st != NB_OK) return st;
    // the ticket must start at zero; the partials are all overwritten
    NB_CUDA(cudaMemsetAsync(&s->sc.ticket, 0, sizeof(unsigned int), stream));
    const int grid = (int)m.E;   // one CTA, hence one partial slot, per element
#define CALL(NN)                                                                                   \
    dot_kernel<NN, 0><<<grid, kRedThreads, 0, stream>>>(a, b, nullptr, nullptr, m, s->partials,    \
                                                       &s->sc, out, nullptr, nullptr)
    NB_DISPATCH_N(m.n, CALL)
#undef CALL
    NB_LAUNCH_CHECK("dot_kernel (allocation-free)");
    return NB_OK;
}

}  // namespace nekgb
