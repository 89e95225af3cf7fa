// C ABI entry points of libnekgb: argument checks, context set-up and
// tear-down, error reporting and kernel timing.  The operator, gather-scatter
// and solver kernels live in the other translation units.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <map>
#include <string.h>

#include <atomic>
#include <new>
#include <string>

#include "internal.cuh"

namespace nekgb {

static thread_local std::string g_last_error;
static std::atomic<long> g_alloc_count{0};

void set_error(const std::string &msg) { g_last_error = msg; }

nb_status fail(nb_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

nb_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
}

nb_status smem_attr(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;   // largest size set
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto it = done.find({kernel, dev});
    if (it != done.end() && it->second >= bytes) return NB_OK;
    NB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done[{kernel, dev}] = bytes;
    return NB_OK;
}

int device_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    cudaGetDevice(&dev);
    int v = dev >= 0 && dev < kMaxDev ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    if (dev >= 0 && dev < kMaxDev) cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    long k = ++g_alloc_count;
    const char *inj = getenv("NEKGB_FAIL_ALLOC");
    if (inj && atol(inj) == k) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes ? bytes : 16);
}

LaunchTimer::LaunchTimer(nb_ctx *ctx, int k) : c(ctx), kid(k) {
    if (c->capturing) {   // counted when the graph is launched
        c->capture_count++;
        return;
    }
    c->n_launched++;
    if (!c->timing) return;
    if (c->event_pool.size() < 2) {
        for (int q = 0; q < 64; q++) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) break;
            c->event_pool.push_back(ev);
        }
    }
    if (c->event_pool.size() < 2) return;
    a = c->event_pool.back(); c->event_pool.pop_back();
    b = c->event_pool.back(); c->event_pool.pop_back();
    cudaEventRecord(a, c->stream);
}

LaunchTimer::~LaunchTimer() {
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->pending.push_back(TimingRec{kid, a, b});
}

nb_status harvest_timing(nb_ctx *c) {
    if (c->pending.empty()) return NB_OK;
    NB_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &r : c->pending) {
        float ms = 0.f;
        NB_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        c->t_ms[r.kid] += ms;
        c->t_launch[r.kid] += 1;
        c->event_pool.push_back(r.a);
        c->event_pool.push_back(r.b);
    }
    c->pending.clear();
    return NB_OK;
}

nb_status check_mesh(nb_box mesh, int n) {
    if (n < 2 || n > kMaxN) return fail(NB_ERR_ARG, "n must be in 2..16");
    if (mesh.ex < 1 || mesh.ey < 1 || mesh.ez < 1)
        return fail(NB_ERR_ARG, "mesh dimensions must be >= 1");
    int64_t E = (int64_t)mesh.ex * mesh.ey * mesh.ez;
    int64_t npts = E * n * n * n;
    if (npts >= ((int64_t)1 << 40)) return fail(NB_ERR_ARG, "mesh too large");
    return NB_OK;
}

static bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

// Whole-box operations that a slab context (nb_setup_slab) cannot do alone:
// its interface nodes also have copies in the neighbouring slabs.
static const char *const slab_refusal =
    "a slab context covers part of the box: use the partitioned solve (nb_slab_* and an exchange between slabs)";

void free_ctx(nb_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *ptrs[] = {c->d_D, c->d_gxyz, c->d_mask, c->d_Df, c->d_gxyz_df, c->d_gxyz32, c->d_minv,
                    c->d_r, c->d_p, c->d_w, c->d_x, c->d_partials, c->d_sc, c->d_hist,
                    c->d_r32, c->d_p32, c->d_w32, c->d_z32};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->cg_graph) cudaGraphExecDestroy(c->cg_graph);
    if (c->cg_graph32) cudaGraphExecDestroy(c->cg_graph32);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto ev : c->event_pool) cudaEventDestroy(ev);
    delete c;
}

nb_status new_ctx(nb_ctx **out, nb_box mesh, int n, nb_precision prec, void *stream) {
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return fail(NB_ERR_OOM, "host allocation of the context failed");
    c->m = make_box_mesh(mesh.ex, mesh.ey, mesh.ez, n);
    c->prec = prec;
    c->stream = (cudaStream_t)stream;
    c->ax_variant = 0;
    {
        const char *st = getenv("NEKGB_F32_STAGED");
        c->f32_plain = st && st[0] == '0';
        // tests of the bounded-wait path: the staged FP32 head's first wait
        // runs out after this many nanoseconds (0 or unset: normal waits)
        const char *tw = getenv("NEKGB_TEST_UNARMED_WAIT_NS");
        c->test_unarmed_wait_ns = tw ? strtoull(tw, nullptr, 10) : 0ull;
        // tests of the exact <w,p>_c sum's range check: shift its scale
        const char *ds = getenv("NEKGB_TEST_DOT_SHIFT");
        c->test_dot_shift = ds ? atoi(ds) : 0;
    }
    *out = c;
    return NB_OK;
}

}  // namespace nekgb

using namespace nekgb;

#define NB_GUARD_BEGIN try {
#define NB_GUARD_END                                                     \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        return fail(NB_ERR_OOM, "host allocation failed");               \
    }                                                                    \
    catch (...) {                                                        \
        return fail(NB_ERR_STATE, "unexpected C++ exception");           \
    }

extern "C" {

const char *nb_status_str(nb_status s) {
    switch (s) {
        case NB_OK: return "NB_OK";
        case NB_ERR_ARG: return "NB_ERR_ARG";
        case NB_ERR_CUDA: return "NB_ERR_CUDA";
        case NB_ERR_OOM: return "NB_ERR_OOM";
        case NB_ERR_NOT_CONVERGED: return "NB_ERR_NOT_CONVERGED";
        case NB_ERR_BREAKDOWN: return "NB_ERR_BREAKDOWN";
        case NB_ERR_TIMEOUT: return "NB_ERR_TIMEOUT";
        case NB_ERR_STATE: return "NB_ERR_STATE";
    }
    return "NB_UNKNOWN";
}

const char *nb_last_error(void) { return g_last_error.c_str(); }

nb_status nb_setup(nb_ctx **out, nb_box mesh, int n, const double *D, const double *gxyz,
                   const uint8_t *mask, nb_precision prec, void *cuda_stream) {
    NB_GUARD_BEGIN
    if (!out) return fail(NB_ERR_ARG, "out is NULL");
    *out = nullptr;
    nb_status s = check_mesh(mesh, n);
    if (s != NB_OK) return s;
    if (!D || !gxyz) return fail(NB_ERR_ARG, "D and gxyz are required");
    if (prec != NB_FP64 && prec != NB_MIXED) return fail(NB_ERR_ARG, "unknown precision");
    nb_ctx *c = nullptr;
    if ((s = new_ctx(&c, mesh, n, prec, cuda_stream)) != NB_OK) return s;
    const int64_t n3 = (int64_t)n * n * n;
    auto bail = [&](nb_status st) { free_ctx(c); return st; };
    memcpy(c->D_host, D, sizeof(double) * n * n);
    cudaError_t e;
    if ((e = dev_alloc((void **)&c->d_D, sizeof(double) * n * n)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc D"));
    if ((e = dev_alloc((void **)&c->d_gxyz, sizeof(double) * 6 * n3 * c->m.E)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc gxyz"));
    c->device_bytes += sizeof(double) * (n * n + 6 * n3 * c->m.E);
    if ((e = cudaMemcpyAsync(c->d_D, D, sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "copy D"));
    if ((e = cudaMemcpyAsync(c->d_gxyz, gxyz, sizeof(double) * 6 * n3 * c->m.E,
                             cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "copy gxyz"));
    if (mask) {
        if ((e = dev_alloc((void **)&c->d_mask, c->m.npts)) != cudaSuccess)
            return bail(cuda_fail(e, "alloc mask"));
        c->device_bytes += c->m.npts;
        if ((e = cudaMemcpyAsync(c->d_mask, mask, c->m.npts, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return bail(cuda_fail(e, "copy mask"));
    }
    if ((s = prepare_df(c)) != NB_OK) return bail(s);
    if (prec == NB_MIXED && (s = prepare_fp32(c)) != NB_OK) return bail(s);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(e, "setup sync"));
    *out = c;
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_setup_box(nb_ctx **out, nb_box mesh, int n, double amp, const double *s3,
                       nb_precision prec, void *cuda_stream) {
    NB_GUARD_BEGIN
    if (!out) return fail(NB_ERR_ARG, "out is NULL");
    *out = nullptr;
    nb_status s = check_mesh(mesh, n);
    if (s != NB_OK) return s;
    if (!s3) return fail(NB_ERR_ARG, "s (3 perturbation coefficients) is required");
    if (prec != NB_FP64 && prec != NB_MIXED) return fail(NB_ERR_ARG, "unknown precision");
    nb_ctx *c = nullptr;
    if ((s = new_ctx(&c, mesh, n, prec, cuda_stream)) != NB_OK) return s;
    auto bail = [&](nb_status st) { free_ctx(c); return st; };
    const int64_t n3 = (int64_t)n * n * n;
    double xi[kMaxN], w[kMaxN];
    if ((s = host_gll(n, xi, w)) != NB_OK) return bail(s);
    if ((s = host_dmat(n, xi, c->D_host)) != NB_OK) return bail(s);
    cudaError_t e;
    if ((e = dev_alloc((void **)&c->d_D, sizeof(double) * n * n)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc D"));
    if ((e = dev_alloc((void **)&c->d_gxyz, sizeof(double) * 6 * n3 * c->m.E)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc gxyz"));
    c->device_bytes += sizeof(double) * (n * n + 6 * n3 * c->m.E);
    if ((e = cudaMemcpyAsync(c->d_D, c->D_host, sizeof(double) * n * n, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "copy D"));
    c->is_box = true;
    c->box_amp = amp;
    c->box_s[0] = s3[0]; c->box_s[1] = s3[1]; c->box_s[2] = s3[2];
    int *d_bad = nullptr;
    if ((e = dev_alloc((void **)&d_bad, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "alloc flag"));
    cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    s = launch_box_geometry(c, amp, s3, d_bad);
    int bad = 0;
    if (s == NB_OK) {
        e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "geometry");
    }
    cudaFree(d_bad);
    if (s != NB_OK) return bail(s);
    if (bad) return bail(fail(NB_ERR_ARG, "the perturbed map folds: |J| <= 0 somewhere"));
    if ((s = prepare_df(c)) != NB_OK) return bail(s);
    if (prec == NB_MIXED && (s = prepare_fp32(c)) != NB_OK) return bail(s);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(e, "setup sync"));
    *out = c;
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_destroy(nb_ctx *ctx) {
    NB_GUARD_BEGIN
    free_ctx(ctx);
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_get_info(const nb_ctx *c, nb_info *info) {
    if (!c || !info) return fail(NB_ERR_ARG, "NULL argument");
    info->ex = c->m.ex; info->ey = c->m.ey; info->ez = c->m.ez; info->n = c->m.n;
    info->nelt = c->m.E;
    info->npts = c->m.npts;
    info->nunique = c->m.NX * c->m.NY * c->m.NZ;
    info->precision = (int)c->prec;
    info->ax_variant = c->ax_variant;
    info->device_bytes = c->device_bytes;
    return NB_OK;
}

nb_status nb_ax(nb_ctx *c, const double *u, double *w) {
    NB_GUARD_BEGIN
    if (!c || !u || !w) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8(u) || !aligned8(w)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    const size_t bytes = sizeof(double) * c->m.npts;
    if ((const char *)u < (const char *)w + bytes && (const char *)w < (const char *)u + bytes)
        return fail(NB_ERR_ARG, "u and w overlap");
    return launch_ax(c, u, w);
    NB_GUARD_END
}

nb_status nb_dssum(nb_ctx *c, double *w) {
    NB_GUARD_BEGIN
    if (!c || !w) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8(w)) return fail(NB_ERR_ARG, "w must be 8-byte aligned");
    return launch_dssum(c, w, false);
    NB_GUARD_END
}

nb_status nb_mask(nb_ctx *c, double *w) {
    NB_GUARD_BEGIN
    if (!c || !w) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8(w)) return fail(NB_ERR_ARG, "w must be 8-byte aligned");
    return launch_mask(c, w);
    NB_GUARD_END
}

nb_status nb_apply(nb_ctx *c, const double *u, double *w) {
    NB_GUARD_BEGIN
    if (c && c->slab) return fail(NB_ERR_STATE, slab_refusal);
    nb_status s = nb_ax(c, u, w);
    if (s != NB_OK) return s;
    return launch_dssum(c, w, true);
    NB_GUARD_END
}

nb_status nb_cg_solve(nb_ctx *c, const double *f, double *x, double tol, int maxit, int *iters,
                      double *relres) {
    NB_GUARD_BEGIN
    if (!c || !f || !x) return fail(NB_ERR_ARG, "NULL argument");
    if (c->slab) return fail(NB_ERR_STATE, slab_refusal);
    if (!aligned8(f) || !aligned8(x)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    if (maxit < 0) return fail(NB_ERR_ARG, "maxit must be >= 0");
    const size_t bytes = sizeof(double) * c->m.npts;
    if ((const char *)f < (const char *)x + bytes && (const char *)x < (const char *)f + bytes)
        return fail(NB_ERR_ARG, "f and x overlap");
    if (c->prec == NB_MIXED) return cg_solve_mixed(c, f, x, tol, maxit, iters, relres);
    return cg_solve_fp64(c, f, x, tol, maxit, iters, relres);
    NB_GUARD_END
}

nb_status nb_cg_solve_host(nb_ctx *c, const double *f_host, double *x_host, double tol, int maxit,
                           int *iters, double *relres) {
    NB_GUARD_BEGIN
    if (!c || !f_host || !x_host) return fail(NB_ERR_ARG, "NULL argument");
    if (c->slab) return fail(NB_ERR_STATE, slab_refusal);
    nb_status s = ensure_cg_workspace(c);
    if (s != NB_OK) return s;
    const size_t bytes = sizeof(double) * c->m.npts;
    double *d_f = nullptr, *d_x = nullptr;
    cudaError_t e;
    if ((e = dev_alloc((void **)&d_f, bytes)) != cudaSuccess) return cuda_fail(e, "alloc f");
    if ((e = dev_alloc((void **)&d_x, bytes)) != cudaSuccess) {
        cudaFree(d_f);
        return cuda_fail(e, "alloc x");
    }
    s = NB_OK;
    e = cudaMemcpyAsync(d_f, f_host, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, x_host, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "copy in");
    if (s == NB_OK) s = nb_cg_solve(c, d_f, d_x, tol, maxit, iters, relres);
    if (s == NB_OK || s == NB_ERR_NOT_CONVERGED || s == NB_ERR_BREAKDOWN) {
        e = cudaMemcpyAsync(x_host, d_x, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "copy out");
    }
    cudaFree(d_f);
    cudaFree(d_x);
    return s;
    NB_GUARD_END
}

nb_status nb_cg_history(nb_ctx *c, double *rho_host, int cap, int *count) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    int cnt = c->d_hist ? c->last_iters + 1 : 0;
    if (count) *count = cnt;
    if (rho_host && cap > 0 && cnt > 0) {
        int m = cnt < cap ? cnt : cap;
        if (m > c->hist_cap) m = c->hist_cap;
        NB_CUDA(cudaMemcpyAsync(rho_host, c->d_hist, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
        NB_CUDA(cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_dot_c(nb_ctx *c, const double *a, const double *b, double *out) {
    NB_GUARD_BEGIN
    if (!c || !a || !b || !out) return fail(NB_ERR_ARG, "NULL argument");
    if (c->slab) return fail(NB_ERR_STATE, slab_refusal);
    return dot_c(c, a, b, out);
    NB_GUARD_END
}

nb_status nb_dot_c_noalloc(nb_box mesh, int n, const double *a, const double *b, double *out,
                           void *cuda_stream) {
    NB_GUARD_BEGIN
    nb_status s = check_mesh(mesh, n);
    if (s != NB_OK) return s;
    if (!a || !b || !out) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8(a) || !aligned8(b) || !aligned8(out)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    const Mesh m = make_box_mesh(mesh.ex, mesh.ey, mesh.ez, n);
    return dot_c_noalloc(m, a, b, out, (cudaStream_t)cuda_stream);
    NB_GUARD_END
}

nb_status nb_scatter_unique(nb_ctx *c, const double *g, double *loc) {
    NB_GUARD_BEGIN
    if (!c || !g || !loc) return fail(NB_ERR_ARG, "NULL argument");
    return launch_scatter_unique(c, g, loc);
    NB_GUARD_END
}

nb_status nb_tables(nb_ctx *c, int64_t *gid, int32_t *mult, uint8_t *mask) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    return launch_tables(c, gid, mult, mask);
    NB_GUARD_END
}

nb_status nb_get_operator(nb_ctx *c, double *D_host, double *gxyz_dev) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    const int n = c->m.n;
    if (D_host) memcpy(D_host, c->D_host, sizeof(double) * n * n);
    if (gxyz_dev)
        NB_CUDA(cudaMemcpyAsync(gxyz_dev, c->d_gxyz, sizeof(double) * 6 * (int64_t)n * n * n * c->m.E,
                                cudaMemcpyDeviceToDevice, c->stream));
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_box_coords(nb_ctx *c, double *xyz) {
    NB_GUARD_BEGIN
    if (!c || !xyz) return fail(NB_ERR_ARG, "NULL argument");
    return launch_box_coords(c, xyz);
    NB_GUARD_END
}

nb_status nb_ax_f32(nb_ctx *c, const float *u, float *w) {
    NB_GUARD_BEGIN
    if (!c || !u || !w) return fail(NB_ERR_ARG, "NULL argument");
    if (!c->d_gxyz32) return fail(NB_ERR_STATE, "the FP32 operator needs an NB_MIXED context");
    if (((uintptr_t)u & 3u) || ((uintptr_t)w & 3u)) return fail(NB_ERR_ARG, "pointers must be 4-byte aligned");
    const size_t bytes = sizeof(float) * c->m.npts;
    if ((const char *)u < (const char *)w + bytes && (const char *)w < (const char *)u + bytes)
        return fail(NB_ERR_ARG, "u and w overlap");
    return launch_ax_f32(c, u, w, 0);
    NB_GUARD_END
}

nb_status nb_dssum_f32(nb_ctx *c, float *w) {
    NB_GUARD_BEGIN
    if (!c || !w) return fail(NB_ERR_ARG, "NULL argument");
    if (((uintptr_t)w & 3u)) return fail(NB_ERR_ARG, "w must be 4-byte aligned");
    return launch_dssum32(c, w);
    NB_GUARD_END
}

nb_status nb_set_mixed_params(nb_ctx *c, double inner_tol, int max_outer) {
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (!(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
        return fail(NB_ERR_ARG, "need 0 < inner_tol < 1 and max_outer >= 1");
    c->mixed_inner_tol = inner_tol;
    c->mixed_max_outer = max_outer;
    return NB_OK;
}

nb_status nb_set_preconditioner(nb_ctx *c, int kind) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (kind != 0 && kind != 1) return fail(NB_ERR_ARG, "preconditioner must be 0 (none) or 1 (Jacobi)");
    if (kind == 1 && c->prec == NB_MIXED)
        return fail(NB_ERR_STATE, "the Jacobi preconditioner applies to NB_FP64 contexts");
    return set_preconditioner(c, kind);
    NB_GUARD_END
}

nb_status nb_jacobi_diagonal(nb_ctx *c, double *minv_dev) {
    NB_GUARD_BEGIN
    if (!c || !minv_dev) return fail(NB_ERR_ARG, "NULL argument");
    if (!c->d_minv) return fail(NB_ERR_STATE, "no Jacobi preconditioner set");
    NB_CUDA(cudaMemcpyAsync(minv_dev, c->d_minv, sizeof(double) * c->m.npts, cudaMemcpyDeviceToDevice, c->stream));
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_solve_stats(const nb_ctx *c, int *iters, int *outer) {
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (iters) *iters = c->last_iters;
    if (outer) *outer = c->prec == NB_MIXED ? c->last_outer : 0;
    return NB_OK;
}

nb_status nb_set_ax_variant(nb_ctx *c, int v) {
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (v < 0 || v > 2) return fail(NB_ERR_ARG, "variant must be 0, 1 or 2");
    c->ax_variant = v;
    if (c->cg_graph) {   // the captured iteration embeds the kernel choice
        cudaGraphExecDestroy(c->cg_graph);
        c->cg_graph = nullptr;
    }
    return NB_OK;
}

nb_status nb_timing_enable(nb_ctx *c, int on) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (on < 0 || on > 2) return fail(NB_ERR_ARG, "nb_timing_enable: on is 0, 1 or 2");
    nb_status s = harvest_timing(c);
    c->timing = on;
    c->n_launched = 0;
    for (int k = 0; k < NB_K_COUNT; k++) { c->t_ms[k] = 0; c->t_launch[k] = 0; }
    return s;
    NB_GUARD_END
}

nb_status nb_launch_count(nb_ctx *c, int64_t *launched) {
    NB_GUARD_BEGIN
    if (!c || !launched) return fail(NB_ERR_ARG, "nb_launch_count: NULL argument");
    *launched = c->n_launched;
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_timing_read(nb_ctx *c, int kid, double *ms, int64_t *launches, int reset) {
    NB_GUARD_BEGIN
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (kid < 0 || kid >= NB_K_COUNT) return fail(NB_ERR_ARG, "bad kernel id");
    nb_status s = harvest_timing(c);
    if (s != NB_OK) return s;
    if (ms) *ms = c->t_ms[kid];
    if (launches) *launches = c->t_launch[kid];
    if (reset) {
        for (int k = 0; k < NB_K_COUNT; k++) { c->t_ms[k] = 0; c->t_launch[k] = 0; }
    }
    return NB_OK;
    NB_GUARD_END
}

}  // extern "C"
