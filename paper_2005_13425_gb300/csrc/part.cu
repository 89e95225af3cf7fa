// The box partitioned into slabs of element layers along z, one per GPU or
// rank: the data-parallel form of the operator's second step, which sums
// element results into shared nodes (arXiv 2005.13425 Sec. III; Nekbone
// itself distributes elements with MPI, Sec. I-II).
//
// A slab context holds the element layers z0 .. z1-1 of an Ex x Ey x Ez box:
// device-built geometry at the global coordinates, the Dirichlet mask of
// the global boundary only, and the weights of <a,b>_c from the global
// multiplicities (a node on a slab's top or bottom plane also has copies in
// the neighbouring slab).  ax_e and the slab-local dssum are the ordinary
// kernels on the slab's elements.
//
// Bit-exact interface sums.  dssum adds the copies of a node from +0.0 in
// ascending element order.  Elements are numbered x fastest, so every copy
// in slab k precedes every copy in slab k+1.  The sum over both slabs is
// therefore the lower slab's partial sum continued by the upper slab's
// copies, one at a time:
//   1. each slab forms the partial sums of its top plane from the raw
//      element results (top_partial) and sends them up;
//   2. the upper slab adds each received partial into the first (lowest
//      element) copy of the node (add_bottom): fl(P + b0), never -0;
//   3. the slab-local dssum then continues ((fl(P + b0) + b1) + ...), the
//      same additions in the same order as the single-box dssum;
//   4. the upper slab sends the final values down (bottom_value) and the
//      lower slab writes them to every copy (set_top).
// No step waits on another slab inside a kernel: the exchanges are host-
// ordered copies or collectives between these launches.
//
// Plane buffers hold one value per node of an interface plane,
// (Ex (n-1) + 1) x (Ey (n-1) + 1) doubles, x fastest.
#include <math.h>

#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

nb_status host_gll(int n, double *xi, double *w);
nb_status host_dmat(int n, const double *x, double *D);
nb_status launch_box_geometry(nb_ctx *c, double amp, const double *s, int *bad_dev);
nb_status prepare_df(nb_ctx *c);
nb_status check_mesh(nb_box mesh, int n);
nb_status new_ctx(nb_ctx **out, nb_box mesh, int n, nb_precision prec, void *stream);
void free_ctx(nb_ctx *c);

namespace {

constexpr int kPartThreads = 256;

// Copies of plane node (gx, gy) on an element layer: up to two elements
// along x and two along y, in ascending element order (ey, then ex).
// Returns the number of copies; idx[] are local point offsets.
__device__ __forceinline__ int plane_copies(int64_t gx, int64_t gy, int ezl, int kk, const Mesh &m,
                                            int64_t (&idx)[4]) {
    const int n = m.n, n1 = n - 1;
    int exs[2], is[2], nx = 0;
    int eys[2], js[2], ny = 0;
    const int64_t qx = gx / n1, rx = gx - qx * n1;
    if (rx == 0) {
        if (qx > 0) { exs[nx] = (int)qx - 1; is[nx] = n1; nx++; }
        if (qx < m.ex) { exs[nx] = (int)qx; is[nx] = 0; nx++; }
    } else {
        exs[nx] = (int)qx; is[nx] = (int)rx; nx++;
    }
    const int64_t qy = gy / n1, ry = gy - qy * n1;
    if (ry == 0) {
        if (qy > 0) { eys[ny] = (int)qy - 1; js[ny] = n1; ny++; }
        if (qy < m.ey) { eys[ny] = (int)qy; js[ny] = 0; ny++; }
    } else {
        eys[ny] = (int)qy; js[ny] = (int)ry; ny++;
    }
    const int64_t n3 = (int64_t)n * n * n;
    int c = 0;
    for (int b = 0; b < ny; b++)
        for (int a = 0; a < nx; a++) {
            const int64_t e = exs[a] + (int64_t)m.ex * (eys[b] + (int64_t)m.ey * ezl);
            idx[c++] = e * n3 + is[a] + n * (js[b] + (int64_t)n * kk);
        }
    return c;
}

// MODE 0 top_partial: buf = (+0.0 + c0) + c1 + ... over the top plane.
// MODE 1 add_bottom:  first bottom copy = buf + c0.
// MODE 2 bottom_value: buf = first bottom copy.
// MODE 3 set_top:     every top copy = buf.
template <int MODE>
__global__ void __launch_bounds__(kPartThreads) plane_kernel(double *__restrict__ w, double *__restrict__ buf, Mesh m) {
    const int64_t np = m.NX * m.NY;
    const bool top = MODE == 0 || MODE == 3;
    const int ezl = top ? m.ez - 1 : 0;
    const int kk = top ? m.n - 1 : 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gy = q / m.NX, gx = q - gy * m.NX;
        int64_t idx[4];
        const int c = plane_copies(gx, gy, ezl, kk, m, idx);
        if (MODE == 0) {
            double s = 0.0;
            for (int k = 0; k < c; k++) s = s + w[idx[k]];
            buf[q] = s;
        } else if (MODE == 1) {
            w[idx[0]] = buf[q] + w[idx[0]];
        } else if (MODE == 2) {
            buf[q] = w[idx[0]];
        } else {
            const double v = buf[q];
            for (int k = 0; k < c; k++) w[idx[k]] = v;
        }
    }
}

// Mask of the global boundary: zero on the box's x and y faces, and on the
// z faces that are faces of the whole box (not on a slab interface).
__global__ void slab_mask_kernel(uint8_t *__restrict__ mask, Mesh m, int z0, int ez_global) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t nzg = (int64_t)ez_global * (n - 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const int64_t ex = e % m.ex, ey = (e / m.ex) % m.ey, ez = e / ((int64_t)m.ex * m.ey);
        const int64_t gx = ex * (n - 1) + i, gy = ey * (n - 1) + j, gz = (ez + z0) * (n - 1) + k;
        const bool b = gx == 0 || gx == m.NX - 1 || gy == 0 || gy == m.NY - 1 || gz == 0 || gz == nzg;
        mask[q] = b ? 0 : 1;
    }
}

// Copies of a node along one direction of the global box.
__device__ __forceinline__ int copies_1d(int idx, int64_t e, int64_t ne, int n) {
    if (idx == 0) return e > 0 ? 2 : 1;
    if (idx == n - 1) return e < ne - 1 ? 2 : 1;
    return 1;
}

// Per-CTA sums of a b / multiplicity over the slab's elements (global
// multiplicities), the last CTA adds the partials in CTA order: a fixed
// order for a given launch.
template <int N>
__global__ void __launch_bounds__(kPartThreads)
slab_dot_kernel(const double *__restrict__ a, const double *__restrict__ b, Mesh m, int z0, int ez_global,
                double *partials, unsigned int *ticket, double *out) {
    constexpr int N3 = N * N * N;
    double acc = 0.0;
    for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const int64_t base = e * N3;
        for (int p = threadIdx.x; p < N3; p += kPartThreads) {
            const int i = p % N, j = (p / N) % N, k = p / (N * N);
            const int mu = copies_1d(i, ex, m.ex, N) * copies_1d(j, ey, m.ey, N) * copies_1d(k, ez + z0, ez_global, N);
            const double cw = mu == 1 ? 1.0 : (mu == 2 ? 0.5 : (mu == 4 ? 0.25 : 0.125));
            acc = fma(a[base + p] * cw, b[base + p], acc);
        }
    }
    double v[1] = {acc}, tot[1];
    if (last_block_reduce<1>(v, partials, 0, blockIdx.x, gridDim.x, gridDim.x, ticket, tot) && threadIdx.x == 0)
        *out = tot[0];
}

// y = alpha x + beta y; beta = 0 does not read y (a copy or scale into a
// buffer of any contents).
__global__ void axpby_kernel(double alpha, const double *__restrict__ x, double beta, double *__restrict__ y,
                             int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = beta == 0.0 ? alpha * x[q] : fma(alpha, x[q], beta * y[q]);
}

nb_status plane_op(nb_ctx *c, int mode, double *w, double *buf) {
    const int64_t np = c->m.NX * c->m.NY;
    const int grid = grid_blocks(np, kPartThreads, device_sms() * 4);
    switch (mode) {
        case 0: plane_kernel<0><<<grid, kPartThreads, 0, c->stream>>>(w, buf, c->m); break;
        case 1: plane_kernel<1><<<grid, kPartThreads, 0, c->stream>>>(w, buf, c->m); break;
        case 2: plane_kernel<2><<<grid, kPartThreads, 0, c->stream>>>(w, buf, c->m); break;
        default: plane_kernel<3><<<grid, kPartThreads, 0, c->stream>>>(w, buf, c->m); break;
    }
    NB_LAUNCH_CHECK("plane_kernel");
    return NB_OK;
}

bool aligned8p(const void *p) { return ((uintptr_t)p & 7u) == 0; }

}  // namespace

nb_status ensure_cg_workspace(nb_ctx *c);

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

static nb_status need_slab(nb_ctx *c) {
    if (!c) return fail(NB_ERR_ARG, "NULL context");
    if (!c->slab) return fail(NB_ERR_STATE, "not a slab context (nb_setup_slab)");
    return NB_OK;
}

extern "C" {

nb_status nb_setup_slab(nb_ctx **out, nb_box global, int z0, int z1, int n, double amp, const double *s3,
                        void *cuda_stream) {
    NB_GUARD_BEGIN
    if (!out) return fail(NB_ERR_ARG, "out is NULL");
    *out = nullptr;
    nb_status s = check_mesh(global, n);
    if (s != NB_OK) return s;
    if (!s3) return fail(NB_ERR_ARG, "s (3 perturbation coefficients) is required");
    if (z0 < 0 || z1 > global.ez || z0 >= z1) return fail(NB_ERR_ARG, "slab layers must satisfy 0 <= z0 < z1 <= ez");
    nb_box local = global;
    local.ez = z1 - z0;
    nb_ctx *c = nullptr;
    if ((s = new_ctx(&c, local, n, NB_FP64, cuda_stream)) != NB_OK) return s;
    auto bail = [&](nb_status st) { free_ctx(c); return st; };
    c->slab = true;
    c->slab_z0 = z0;
    c->slab_ez_global = global.ez;
    const int64_t n3 = (int64_t)n * n * n;
    double xi[kMaxN], w[kMaxN];
    if ((s = host_gll(n, xi, w)) != NB_OK) return bail(s);
    if ((s = host_dmat(n, xi, c->D_host)) != NB_OK) return bail(s);
    cudaError_t e;
    if ((e = dev_alloc((void **)&c->d_D, sizeof(double) * n * n)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc D"));
    if ((e = dev_alloc((void **)&c->d_gxyz, sizeof(double) * 6 * n3 * c->m.E)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc gxyz"));
    if ((e = dev_alloc((void **)&c->d_mask, c->m.npts)) != cudaSuccess) return bail(cuda_fail(e, "alloc mask"));
    c->device_bytes += sizeof(double) * (n * n + 6 * n3 * c->m.E) + c->m.npts;
    if ((e = cudaMemcpyAsync(c->d_D, c->D_host, sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "copy D"));
    c->is_box = true;
    c->box_amp = amp;
    c->box_s[0] = s3[0]; c->box_s[1] = s3[1]; c->box_s[2] = s3[2];
    slab_mask_kernel<<<grid_blocks(c->m.npts, kPartThreads, device_sms() * 8), kPartThreads, 0, c->stream>>>(
        c->d_mask, c->m, z0, global.ez);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "slab_mask_kernel"));
    int *d_bad = nullptr;
    if ((e = dev_alloc((void **)&d_bad, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "alloc flag"));
    int bad = 0;
    e = cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    s = e == cudaSuccess ? launch_box_geometry(c, amp, s3, d_bad) : cuda_fail(e, "clear flag");
    if (s == NB_OK) {
        e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "geometry");
    }
    cudaFree(d_bad);
    if (s != NB_OK) return bail(s);
    if (bad) return bail(fail(NB_ERR_ARG, "the perturbed map folds: |J| <= 0 somewhere"));
    if ((s = prepare_df(c)) != NB_OK) return bail(s);
    if ((s = ensure_cg_workspace(c)) != NB_OK) return bail(s);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(e, "setup sync"));
    *out = c;
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_slab_info(nb_ctx *c, int64_t *plane_nodes, int *has_below, int *has_above) {
    nb_status s = need_slab(c);
    if (s != NB_OK) return s;
    if (plane_nodes) *plane_nodes = c->m.NX * c->m.NY;
    if (has_below) *has_below = c->slab_z0 > 0;
    if (has_above) *has_above = c->slab_z0 + c->m.ez < c->slab_ez_global;
    return NB_OK;
}

static nb_status plane_entry(nb_ctx *c, int mode, double *w, double *buf) {
    NB_GUARD_BEGIN
    nb_status s = need_slab(c);
    if (s != NB_OK) return s;
    if (!w || !buf) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8p(w) || !aligned8p(buf)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    return plane_op(c, mode, w, buf);
    NB_GUARD_END
}

nb_status nb_slab_top_partial(nb_ctx *c, const double *w, double *buf) {
    return plane_entry(c, 0, const_cast<double *>(w), buf);
}
nb_status nb_slab_add_bottom(nb_ctx *c, double *w, const double *buf) {
    return plane_entry(c, 1, w, const_cast<double *>(buf));
}
nb_status nb_slab_bottom_value(nb_ctx *c, const double *w, double *buf) {
    return plane_entry(c, 2, const_cast<double *>(w), buf);
}
nb_status nb_slab_set_top(nb_ctx *c, double *w, const double *buf) {
    return plane_entry(c, 3, w, const_cast<double *>(buf));
}

nb_status nb_slab_dot(nb_ctx *c, const double *a, const double *b, double *out_host) {
    NB_GUARD_BEGIN
    nb_status s = need_slab(c);
    if (s != NB_OK) return s;
    if (!a || !b || !out_host) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8p(a) || !aligned8p(b)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    const int64_t cap = (int64_t)device_sms() * 4;
    const int grid = (int)(c->m.E < cap ? c->m.E : cap);
    double *d_out = c->d_partials + c->partial_cap - 1;
#define CALL(NN)                                                                                          \
    case NN:                                                                                              \
        slab_dot_kernel<NN><<<grid, kPartThreads, 0, c->stream>>>(a, b, c->m, c->slab_z0, c->slab_ez_global, \
                                                                  c->d_partials, &c->d_sc->ticket, d_out);  \
        break;
    switch (c->m.n) {
        CALL(2) CALL(3) CALL(4) CALL(5) CALL(6) CALL(7) CALL(8) CALL(9) CALL(10) CALL(11) CALL(12)
        CALL(13) CALL(14) CALL(15) CALL(16)
        default: return fail(NB_ERR_ARG, "unsupported n");
    }
#undef CALL
    NB_LAUNCH_CHECK("slab_dot_kernel");
    NB_CUDA(cudaMemcpyAsync(out_host, d_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    return NB_OK;
    NB_GUARD_END
}

nb_status nb_axpby(nb_ctx *c, double alpha, const double *x, double beta, double *y) {
    NB_GUARD_BEGIN
    if (!c || !x || !y) return fail(NB_ERR_ARG, "NULL argument");
    if (!aligned8p(x) || !aligned8p(y)) return fail(NB_ERR_ARG, "pointers must be 8-byte aligned");
    const int grid = grid_blocks(c->m.npts, kPartThreads, device_sms() * 8);
    axpby_kernel<<<grid, kPartThreads, 0, c->stream>>>(alpha, x, beta, y, c->m.npts);
    NB_LAUNCH_CHECK("axpby_kernel");
    return NB_OK;
    NB_GUARD_END
}

}  // extern "C"
