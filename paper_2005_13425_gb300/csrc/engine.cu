// Batched and served CG solves: many box problems of different sizes and
// polynomial orders advance together, one launch per kernel and per n each
// iteration (the paper's small-problem limit, Sec. VI.B and VII, motivates
// batching: below ~500k DOF a GPU is poorly used by one problem).
//
// * Memory: one device arena, carved by a first-fit allocator; a request is
//   admitted only if its footprint (gxyz pairs + four CG vectors + tile
//   partials) fits in the free space.
// * Work: every problem's elements are split into tiles of `te` elements,
//   its shared nodes into tiles of 2048 nodes.  For each n the active
//   problems' tiles form a device-side list; the kernels stride over the
//   list, so captured CUDA graphs stay valid while problems join and leave.
// * Reductions: each tile writes one partial; the last tile of a problem
//   (per-problem ticket) sums that problem's partials in a fixed order and
//   performs its scalar step.  A problem's arithmetic therefore depends only
//   on the problem, never on what else is in the batch: results are
//   bit-identical alone and in any mix.
// * Autotuning: for each n the first use times the CG head kernel with one
//   or two line tasks per thread and 4, 8 or 16 elements per tile on a
//   synthetic problem, and caches the choice (NEKGB_TUNE_CACHE file).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ax_df_core.cuh"
#include "gs_nodes.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

constexpr int kEngMaxSlots = 1024;
constexpr int kDsTile = 2048;   // shared nodes per dssum tile (256 threads x 8)
constexpr int kEngThreads = 256;

struct ProbDesc {
    Mesh m;
    float2 *g;                  // gxyz pairs [E][6][n^3]
    double *r, *p, *w, *x;      // CG vectors, local storage
    double *partials;           // ntile_ax + ntile_ds slots
    int ntile_ax, ntile_ds, te;
    int cx, cy, cz;
    int pad;
    CgScalars sc;
};

// ---------------------------------------------------------------- kernels
// CG head over a list of (slot, tile) work units.
template <int N, int T>
__global__ void __launch_bounds__(T, (T <= 320 ? 3 : 1))
eng_ax_head(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles,
            const __grid_constant__ DfEo<N> D) {
    constexpr int N3 = N * N * N;
    extern __shared__ float2 sm[];
    __shared__ int s_emax;
    __shared__ double red[32];
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.sc.done) continue;                     // uniform over the CTA
        const double beta = P.sc.it == 0 ? 0.0 : P.sc.beta;
        const double xa = P.sc.x_alpha;
        const Mesh m = P.m;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
        double dot = 0.0;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t eb = e * N3;
            DfElemIO io;
            io.u = nullptr;
            io.r = P.r + eb;
            io.p = P.p + eb;
            io.x = P.x + eb;
            io.minv = nullptr;
            io.w = P.w + eb;
            io.g = P.g + e * 6 * N3;
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            df_element<N, 1, true, T>(io, beta, xa, true, 1023, m, ex, ey, ez, D, sm, &s_emax, dot);
        }
        const double b = block_sum(dot, red);
        if (threadIdx.x == 0) P.partials[tile.y] = b;
    }
}

// dssum of w over (slot, node tile) work units, shared-node <w,p>_c, and in
// the problem's last tile: alpha = rho/<w,p>_c.
__global__ void __launch_bounds__(kEngThreads)
eng_dssum(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles) {
    __shared__ double red[32];
    __shared__ int s_last;
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.sc.done) continue;
        const Mesh m = P.m;
        const int total = P.cx + P.cy + P.cz;
        double *w = P.w;
        const double *p = P.p;
        double dot = 0.0;
        const int q0 = tile.y * kDsTile;
        const int q1 = q0 + kDsTile < total ? q0 + kDsTile : total;
        for (int q = q0 + threadIdx.x; q < q1; q += kEngThreads) {
            int gx, gy, gz;
            shared_node(q, m, P.cx, P.cy, gx, gy, gz);
            int64_t idx[8];
            const int c = node_copies(gx, gy, gz, m, idx);
            double s;
            double ps;
            int lg;
            if (c == 2) {
                s = plus_zero(w[idx[0]]) + w[idx[1]];
                ps = p[idx[0]] + p[idx[1]];
                lg = 1;
            } else if (c == 4) {
                double a[4];
#pragma unroll
                for (int k = 0; k < 4; k++) a[k] = w[idx[k]];
                s = plus_zero(a[0]);
#pragma unroll
                for (int k = 1; k < 4; k++) s = s + a[k];
                ps = p[idx[0]];
#pragma unroll
                for (int k = 1; k < 4; k++) ps += p[idx[k]];
                lg = 2;
            } else {
                double a[8];
#pragma unroll
                for (int k = 0; k < 8; k++) a[k] = w[idx[k]];
                s = plus_zero(a[0]);
#pragma unroll
                for (int k = 1; k < 8; k++) s = s + a[k];
                ps = p[idx[0]];
#pragma unroll
                for (int k = 1; k < 8; k++) ps += p[idx[k]];
                lg = 3;
            }
            for (int k = 0; k < c; k++) w[idx[k]] = s;
            dot = node_dot(dot, s, lg, ps);
        }
        const double b = block_sum(dot, red);
        if (threadIdx.x == 0) {
            P.partials[P.ntile_ax + tile.y] = b;
            __threadfence();
            const unsigned t = atomicAdd(&P.sc.ticket, 1u);
            s_last = (t == (unsigned)P.ntile_ds - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double acc = 0.0;
            const int cnt = P.ntile_ax + P.ntile_ds;
            for (int k = threadIdx.x; k < cnt; k += kEngThreads) acc += __ldcg(P.partials + k);
            const double pap = block_sum(acc, red);
            if (threadIdx.x == 0) {
                P.sc.ticket = 0;
                P.sc.pap = pap;
                if (!(pap > 0.0) || !isfinite(pap)) {
                    P.sc.status = (int)NB_ERR_BREAKDOWN;
                    P.sc.done = 1;
                    P.sc.x_alpha = 0.0;
                } else {
                    P.sc.alpha = P.sc.rho / pap;
                    P.sc.x_alpha = P.sc.alpha;
                }
            }
        }
        __syncthreads();
    }
}

// r -= alpha w with <r,r>_c per tile; the problem's last tile forms rho,
// beta and the convergence decision.
template <int N>
__global__ void __launch_bounds__(kEngThreads)
eng_update(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles) {
    constexpr int N3 = N * N * N;
    __shared__ double red[32];
    __shared__ int s_last;
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.sc.done) continue;
        const Mesh m = P.m;
        const double alpha = P.sc.alpha;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
        double acc = 0.0;
        for (int64_t e = e0; e < e1; e++) {
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            double *r = P.r + e * N3;
            const double *w = P.w + e * N3;
#pragma unroll 4
            for (int q = threadIdx.x; q < N3; q += kEngThreads) {
                const int i = q % N, j = (q / N) % N, k = q / (N * N);
                const double rn = fma(-alpha, w[q], r[q]);
                r[q] = rn;
                acc = fma(scale_down_pow2(rn, log2_mult(i, j, k, ex, ey, ez, m)), rn, acc);
            }
        }
        const double b = block_sum(acc, red);
        if (threadIdx.x == 0) {
            P.partials[tile.y] = b;
            __threadfence();
            const unsigned t = atomicAdd(&P.sc.ticket, 1u);
            s_last = (t == (unsigned)P.ntile_ax - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double a2 = 0.0;
            for (int k = threadIdx.x; k < P.ntile_ax; k += kEngThreads) a2 += __ldcg(P.partials + k);
            const double rho = block_sum(a2, red);
            if (threadIdx.x == 0) {
                P.sc.ticket = 0;
                P.sc.rho_old = P.sc.rho;
                P.sc.rho = rho;
                P.sc.beta = rho / P.sc.rho_old;
                const int it = P.sc.it + 1;
                P.sc.it = it;
                const bool conv = P.sc.tol > 0.0 && sqrt(rho) / sqrt(P.sc.fnorm2) <= P.sc.tol;
                if (rho == 0.0 || conv || it >= P.sc.maxit) P.sc.done = 1;
            }
        }
        __syncthreads();
    }
}

// Start of one problem's solve (x0 = 0, so r = f): p = 0, x = 0 and
// rho = <r,r>_c = <f,f>_c; one CTA per element tile of that problem.
template <int N>
__global__ void __launch_bounds__(kEngThreads) eng_start(ProbDesc *__restrict__ desc, int slot) {
    constexpr int N3 = N * N * N;
    __shared__ double red[32];
    __shared__ int s_last;
    ProbDesc &P = desc[slot];
    const Mesh m = P.m;
    const int64_t e0 = (int64_t)blockIdx.x * P.te;
    const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
    double acc = 0.0;
    for (int64_t e = e0; e < e1; e++) {
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const double *r = P.r + e * N3;
        for (int q = threadIdx.x; q < N3; q += kEngThreads) {
            const int i = q % N, j = (q / N) % N, k = q / (N * N);
            P.p[e * N3 + q] = 0.0;
            P.x[e * N3 + q] = 0.0;
            const double rv = r[q];
            acc = fma(scale_down_pow2(rv, log2_mult(i, j, k, ex, ey, ez, m)), rv, acc);
        }
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0) {
        P.partials[blockIdx.x] = b;
        __threadfence();
        const unsigned t = atomicAdd(&P.sc.ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kEngThreads) a2 += __ldcg(P.partials + k);
    const double rho = block_sum(a2, red);
    if (threadIdx.x == 0) {
        P.sc.ticket = 0;
        P.sc.rho = rho;
        P.sc.rho_old = 1.0;
        P.sc.fnorm2 = rho;
        P.sc.beta = 0.0;
        P.sc.x_alpha = 0.0;
        P.sc.it = 0;
        P.sc.status = 0;
        P.sc.done = (rho == 0.0 || P.sc.maxit == 0) ? 1 : 0;
    }
}

// r = mask(Q fu): a field given per unique node (x fastest) copied to every
// local copy, zero on the faces of the box (the right-hand side of a request
// submitted in unique-node form).
__global__ void eng_scatter_mask(ProbDesc *__restrict__ desc, int slot, const double *__restrict__ fu) {
    const ProbDesc &P = desc[slot];
    const Mesh m = P.m;
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        int ex, ey, ez;
        element_coords(e, m, ex, ey, ez);
        const int64_t gx = (int64_t)ex * (n - 1) + i, gy = (int64_t)ey * (n - 1) + j,
                      gz = (int64_t)ez * (n - 1) + k;
        P.r[q] = on_box_face(i, j, k, ex, ey, ez, m) ? 0.0 : fu[gx + m.NX * (gy + m.NY * gz)];
    }
}

// x += x_alpha p for one problem (the update owed by its last iteration).
__global__ void eng_final_x(ProbDesc *__restrict__ desc, int slot) {
    ProbDesc &P = desc[slot];
    const double xa = P.sc.x_alpha;
    if (xa == 0.0) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.m.npts;
         q += (int64_t)gridDim.x * blockDim.x)
        P.x[q] = fma(xa, P.p[q], P.x[q]);
}

}  // namespace nekgb

// ---------------------------------------------------------------- host side
namespace nekgb {

// First-fit device arena with coalescing free list (offsets in bytes).
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    static size_t align(size_t b) { return (b + 255) & ~(size_t)255; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align(bytes);
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct EngSlot {
    bool used = false;
    int n = 0;
    size_t off = 0, bytes = 0;
    double t_submit = 0.0;
};

struct NGroup {
    int lpt = 0, te = 0;                 // tuned (0: not yet)
    int2 *d_ax = nullptr, *d_ds = nullptr;
    int *d_cnt = nullptr;                // [0] = ax tiles, [1] = dssum tiles
    int cap_ax = 0, cap_ds = 0;
    std::vector<int> slots;
    bool dirty = false;
    double D[kMaxN * kMaxN];
};

}  // namespace nekgb

struct nb_engine {
    cudaStream_t stream = nullptr;
    nekgb::Arena arena;
    nekgb::ProbDesc *d_desc = nullptr, *h_desc = nullptr;
    nekgb::EngSlot slots[nekgb::kEngMaxSlots];
    nekgb::NGroup groups[nekgb::kMaxN + 1];
    cudaGraphExec_t graph = nullptr;
    unsigned graph_key = 0;
    int graph_chunk = 0;
    int sms = 1;
};

namespace nekgb {

static size_t desc_footprint(const Mesh &m, int te, size_t *parts) {
    const int64_t n3 = (int64_t)m.n * m.n * m.n;
    int cx, cy, cz;
    shared_counts(m, cx, cy, cz);
    const int64_t ntax = (m.E + te - 1) / te;
    const int64_t total = (int64_t)cx + cy + cz;
    const int64_t ntds = total > 0 ? (total + kDsTile - 1) / kDsTile : 1;
    parts[0] = Arena::align(sizeof(float2) * 6 * n3 * m.E);          // gxyz pairs
    parts[1] = Arena::align(sizeof(double) * m.npts);                 // each CG vector
    parts[2] = Arena::align(sizeof(double) * (ntax + ntds + 1));      // partials
    return parts[0] + 4 * parts[1] + parts[2];
}

static Mesh make_mesh(nb_box b, int n) {
    Mesh m;
    m.ex = b.ex; m.ey = b.ey; m.ez = b.ez; m.n = n;
    m.E = (int64_t)b.ex * b.ey * b.ez;
    m.npts = m.E * n * n * n;
    m.NX = (int64_t)b.ex * (n - 1) + 1;
    m.NY = (int64_t)b.ey * (n - 1) + 1;
    m.NZ = (int64_t)b.ez * (n - 1) + 1;
    return m;
}

// ---- kernel dispatch over (N, LPT)
template <int N, int LPT>
static nb_status head_launch(nb_engine *g, const NGroup &G) {
    constexpr int T = df_threads_lpt(N, LPT);
    const size_t smem = sizeof(float2) * 6 * N * N * N;
    static bool configured = false;
    if (!configured) {
        NB_CUDA(cudaFuncSetAttribute(eng_ax_head<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_ax_head<N, T>, T, smem);
    if (occ < 1) occ = 1;
    DfEo<N> D;
    eo_consts<N>(G.D, false, D.fwd);
    eo_consts<N>(G.D, true, D.bwd);
    eng_ax_head<N, T><<<g->sms * occ, T, smem, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt, D);
    NB_LAUNCH_CHECK("eng_ax_head");
    return NB_OK;
}

template <int N>
static nb_status group_iteration(nb_engine *g, const NGroup &G) {
    nb_status s;
    if constexpr (N >= 13) s = head_launch<N, 2>(g, G);
    else s = G.lpt == 2 ? head_launch<N, 2>(g, G) : head_launch<N, 1>(g, G);
    if (s != NB_OK) return s;
    eng_dssum<<<g->sms * 8, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ds, G.d_cnt + 1);
    NB_LAUNCH_CHECK("eng_dssum");
    eng_update<N><<<g->sms * 4, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt);
    NB_LAUNCH_CHECK("eng_update");
    return NB_OK;
}

static nb_status dispatch_iteration(nb_engine *g, int n) {
    const NGroup &G = g->groups[n];
    switch (n) {
#define NB_CASE(NN) case NN: return group_iteration<NN>(g, G);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
}

static nb_status dispatch_start(nb_engine *g, int n, int slot, int grid) {
    switch (n) {
#define NB_CASE(NN) case NN: eng_start<NN><<<grid, kEngThreads, 0, g->stream>>>(g->d_desc, slot); break;
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
        default: return fail(NB_ERR_ARG, "unsupported n");
    }
    NB_LAUNCH_CHECK("eng_start");
    return NB_OK;
}

// ---- autotuner: lines per thread and elements per tile, per n
static std::mutex g_tune_mu;

static std::string tune_cache_path() {
    const char *p = getenv("NEKGB_TUNE_CACHE");
    return p ? std::string(p) : std::string();
}

static bool tune_lookup(const std::string &key, int *lpt, int *te) {
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char k[512];
    int a, b;
    bool found = false;
    while (fscanf(f, "%511s %d %d", k, &a, &b) == 3)
        if (key == k) { *lpt = a; *te = b; found = true; }
    fclose(f);
    return found;
}

static void tune_store(const std::string &key, int lpt, int te) {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), lpt, te);
    fclose(f);
}

nb_status engine_submit_internal(nb_engine *g, nb_box box, int n, double amp, const double *s3,
                                 double tol, int maxit, const double *f, int te, int *id,
                                 bool f_unique = false);
nb_status engine_retire_internal(nb_engine *g, int id, double *x);
nb_status engine_step_internal(nb_engine *g, int iters);

// Time the CG iteration of a synthetic 8x8x8-element problem for each
// candidate (lines per thread, elements per tile) and keep the fastest.
static nb_status autotune(nb_engine *g, int n) {
    NGroup &G = g->groups[n];
    if (G.lpt) return NB_OK;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char key[512];
    snprintf(key, sizeof key, "n%d_fp64_sm%d_%.200s", n, prop.multiProcessorCount, prop.name);
    for (char *c = key; *c; c++)
        if (*c == ' ') *c = '_';
    int lpt = 0, te = 0;
    if (tune_lookup(key, &lpt, &te)) {
        G.lpt = lpt;
        G.te = te;
        return NB_OK;
    }
    const int lpts[2] = {1, 2};
    const int tes[3] = {4, 8, 16};
    float best = 1e30f;
    int bl = n >= 13 ? 2 : 1, bt = 8;
    const nb_box box = {8, 8, 8};
    const Mesh m = make_mesh(box, n);
    double *f = nullptr;
    cudaError_t e = dev_alloc((void **)&f, sizeof(double) * m.npts);
    if (e != cudaSuccess) return cuda_fail(e, "alloc tuning rhs");
    cudaMemsetAsync(f, 0, sizeof(double) * m.npts, g->stream);
    const double s3[3] = {0.3, -0.5, 0.7};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    nb_status st = NB_OK;
    for (int li = 0; li < 2 && st == NB_OK; li++) {
        if (n >= 13 && lpts[li] == 1) continue;
        for (int ti = 0; ti < 3 && st == NB_OK; ti++) {
            G.lpt = lpts[li];
            if (g->graph) {   // captured with another candidate's kernels
                cudaGraphExecDestroy(g->graph);
                g->graph = nullptr;
                g->graph_key = 0;
            }
            int id = -1;
            // the rhs is made nonzero by setting one value: rho > 0
            const double one = 1.0;
            cudaMemcpyAsync(f + m.npts / 2, &one, sizeof(double), cudaMemcpyHostToDevice, g->stream);
            st = engine_submit_internal(g, box, n, 0.05, s3, 0.0, 1 << 30, f, tes[ti], &id);
            if (st == NB_ERR_OOM) {   // no room for the tuning problem: keep the defaults
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                cudaFree(f);
                G.lpt = n >= 13 ? 2 : 1;
                G.te = 8;
                return NB_OK;
            }
            if (st != NB_OK) break;
            st = engine_step_internal(g, 2);                       // warm-up
            cudaEventRecord(a, g->stream);
            if (st == NB_OK) st = engine_step_internal(g, 8);
            cudaEventRecord(b, g->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) { best = ms; bl = lpts[li]; bt = tes[ti]; }
            nb_status s2 = engine_retire_internal(g, id, nullptr);
            if (st == NB_OK) st = s2;
        }
    }
    cudaStreamSynchronize(g->stream);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(f);
    if (g->graph) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
        g->graph_key = 0;
    }
    G.lpt = bl;
    G.te = bt;
    if (st == NB_OK) tune_store(key, bl, bt);
    return st;
}

static nb_status ensure_group(nb_engine *g, int n, int64_t max_tiles_ax, int64_t max_tiles_ds) {
    NGroup &G = g->groups[n];
    if (!G.d_cnt) {
        double xi[kMaxN], w[kMaxN];
        nb_status s = host_gll(n, xi, w);
        if (s != NB_OK) return s;
        if ((s = host_dmat(n, xi, G.D)) != NB_OK) return s;
        cudaError_t e = dev_alloc((void **)&G.d_cnt, 2 * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "alloc tile counts");
        NB_CUDA(cudaMemsetAsync(G.d_cnt, 0, 2 * sizeof(int), g->stream));
    }
    auto grow = [&](int2 **arr, int *cap, int64_t need) -> nb_status {
        if (need <= *cap) return NB_OK;
        int64_t nc = need < 4096 ? 4096 : need * 2;
        int2 *na = nullptr;
        cudaError_t e = dev_alloc((void **)&na, sizeof(int2) * nc);
        if (e != cudaSuccess) return cuda_fail(e, "alloc tile list");
        if (*arr) {
            cudaStreamSynchronize(g->stream);
            cudaFree(*arr);
        }
        *arr = na;
        *cap = (int)nc;
        if (g->graph) {   // the captured graph refers to the old list
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
            g->graph_key = 0;
        }
        return NB_OK;
    };
    nb_status s = grow(&G.d_ax, &G.cap_ax, max_tiles_ax);
    if (s != NB_OK) return s;
    return grow(&G.d_ds, &G.cap_ds, max_tiles_ds);
}

// Rebuild the device tile lists of the groups whose membership changed.
static nb_status refresh_tiles(nb_engine *g) {
    for (int n = 2; n <= kMaxN; n++) {
        NGroup &G = g->groups[n];
        if (!G.dirty) continue;
        std::vector<int2> ax, ds;
        for (int slot : G.slots) {
            const ProbDesc &P = g->h_desc[slot];
            for (int j = 0; j < P.ntile_ax; j++) ax.push_back(make_int2(slot, j));
            for (int j = 0; j < P.ntile_ds; j++) ds.push_back(make_int2(slot, j));
        }
        nb_status s = ensure_group(g, n, (int64_t)ax.size(), (int64_t)ds.size());
        if (s != NB_OK) return s;
        if (!ax.empty())
            NB_CUDA(cudaMemcpyAsync(G.d_ax, ax.data(), sizeof(int2) * ax.size(), cudaMemcpyHostToDevice, g->stream));
        if (!ds.empty())
            NB_CUDA(cudaMemcpyAsync(G.d_ds, ds.data(), sizeof(int2) * ds.size(), cudaMemcpyHostToDevice, g->stream));
        int cnt[2] = {(int)ax.size(), (int)ds.size()};
        NB_CUDA(cudaMemcpyAsync(G.d_cnt, cnt, sizeof cnt, cudaMemcpyHostToDevice, g->stream));
        NB_CUDA(cudaStreamSynchronize(g->stream));   // cnt lives on the host stack
        G.dirty = false;
    }
    return NB_OK;
}

nb_status engine_submit_internal(nb_engine *g, nb_box box, int n, double amp, const double *s3,
                                 double tol, int maxit, const double *f, int te, int *id,
                                 bool f_unique) {
    const Mesh m = make_mesh(box, n);
    size_t parts[3];
    const size_t bytes = desc_footprint(m, te, parts);
    int slot = -1;
    for (int k = 0; k < kEngMaxSlots; k++)
        if (!g->slots[k].used) { slot = k; break; }
    if (slot < 0) return fail(NB_ERR_OOM, "engine: all request slots are in use");
    size_t off = 0;
    if (!g->arena.alloc(bytes, &off))
        return fail(NB_ERR_OOM, "engine: the request's footprint does not fit in the free arena");
    // ensure the group exists (D, counts) before building the problem
    nb_status s = ensure_group(g, n, 0, 0);
    if (s != NB_OK) { g->arena.release(off, bytes); return s; }
    char *base = g->arena.base + off;
    ProbDesc &P = g->h_desc[slot];
    memset(&P, 0, sizeof P);
    P.m = m;
    P.g = (float2 *)base;
    P.r = (double *)(base + parts[0]);
    P.p = (double *)(base + parts[0] + parts[1]);
    P.w = (double *)(base + parts[0] + 2 * parts[1]);
    P.x = (double *)(base + parts[0] + 3 * parts[1]);
    P.partials = (double *)(base + parts[0] + 4 * parts[1]);
    P.te = te;
    shared_counts(m, P.cx, P.cy, P.cz);
    P.ntile_ax = (int)((m.E + te - 1) / te);
    const int64_t total = (int64_t)P.cx + P.cy + P.cz;
    P.ntile_ds = total > 0 ? (int)((total + kDsTile - 1) / kDsTile) : 1;
    P.sc.tol = tol;
    P.sc.maxit = maxit;
    P.sc.done = 1;   // not iterated until the start kernel has run
    cudaError_t e;
    if ((e = cudaMemcpyAsync(g->d_desc + slot, &P, sizeof(ProbDesc), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess) {
        g->arena.release(off, bytes);
        return cuda_fail(e, "engine: descriptor upload");
    }
    int *d_bad = (int *)(P.partials);   // scratch: the partials are rewritten by the start kernel
    NB_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), g->stream));
    s = launch_box_geometry_pairs(m, amp, s3, g->groups[n].D, P.g, d_bad, g->stream);
    if (s == NB_OK && !f_unique &&
        (e = cudaMemcpyAsync(P.r, f, sizeof(double) * m.npts, cudaMemcpyDeviceToDevice, g->stream)) != cudaSuccess)
        s = cuda_fail(e, "engine: copy rhs");
    if (s == NB_OK && f_unique) {
        eng_scatter_mask<<<grid_blocks(m.npts, 256, g->sms * 8), 256, 0, g->stream>>>(g->d_desc, slot, f);
        if ((e = cudaGetLastError()) != cudaSuccess) s = cuda_fail(e, "eng_scatter_mask");
    }
    int bad = 0;
    if (s == NB_OK && (e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess)
        s = cuda_fail(e, "engine: geometry flag");
    if (s == NB_OK && (e = cudaStreamSynchronize(g->stream)) != cudaSuccess) s = cuda_fail(e, "engine: setup");
    if (s == NB_OK && bad) s = fail(NB_ERR_ARG, "engine: the perturbed map folds (|J| <= 0)");
    if (s == NB_OK) s = dispatch_start(g, n, slot, P.ntile_ax);
    if (s != NB_OK) {
        g->arena.release(off, bytes);
        return s;
    }
    g->slots[slot].used = true;
    g->slots[slot].n = n;
    g->slots[slot].off = off;
    g->slots[slot].bytes = bytes;
    g->groups[n].slots.push_back(slot);
    g->groups[n].dirty = true;
    *id = slot;
    return NB_OK;
}

nb_status engine_step_internal(nb_engine *g, int iters) {
    nb_status s = refresh_tiles(g);
    if (s != NB_OK) return s;
    unsigned key = 0;
    for (int n = 2; n <= kMaxN; n++)
        if (!g->groups[n].slots.empty()) key |= 1u << n;
    if (!key || iters <= 0) return NB_OK;
    const int chunk = 8;
    if (!g->graph || g->graph_key != key || g->graph_chunk != chunk) {
        if (g->graph) {
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
        }
        cudaGraph_t gr = nullptr;
        NB_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < chunk && s == NB_OK; k++)
            for (int n = 2; n <= kMaxN && s == NB_OK; n++)
                if (key & (1u << n)) s = dispatch_iteration(g, n);
        cudaError_t e = cudaStreamEndCapture(g->stream, &gr);
        if (s != NB_OK) {
            if (gr) cudaGraphDestroy(gr);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "engine: end capture");
        e = cudaGraphInstantiate(&g->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(e, "engine: instantiate");
        g->graph_key = key;
        g->graph_chunk = chunk;
    }
    for (int done = 0; done < iters; done += chunk) NB_CUDA(cudaGraphLaunch(g->graph, g->stream));
    // refresh the host mirror of every descriptor's scalars
    NB_CUDA(cudaMemcpyAsync(g->h_desc, g->d_desc, sizeof(ProbDesc) * kEngMaxSlots, cudaMemcpyDeviceToHost, g->stream));
    NB_CUDA(cudaStreamSynchronize(g->stream));
    return NB_OK;
}

nb_status engine_retire_internal(nb_engine *g, int id, double *x) {
    if (id < 0 || id >= kEngMaxSlots || !g->slots[id].used) return fail(NB_ERR_ARG, "engine: unknown request id");
    EngSlot &S = g->slots[id];
    const ProbDesc &P = g->h_desc[id];
    eng_final_x<<<grid_blocks(P.m.npts, 256, g->sms * 8), 256, 0, g->stream>>>(g->d_desc, id);
    NB_LAUNCH_CHECK("eng_final_x");
    if (x) NB_CUDA(cudaMemcpyAsync(x, P.x, sizeof(double) * P.m.npts, cudaMemcpyDeviceToDevice, g->stream));
    // mark inactive on the device before the slot can be reused
    ProbDesc dead = P;
    dead.sc.done = 1;
    NB_CUDA(cudaMemcpyAsync(g->d_desc + id, &dead, sizeof(ProbDesc), cudaMemcpyHostToDevice, g->stream));
    NB_CUDA(cudaStreamSynchronize(g->stream));
    NGroup &G = g->groups[S.n];
    for (size_t k = 0; k < G.slots.size(); k++)
        if (G.slots[k] == id) { G.slots.erase(G.slots.begin() + k); break; }
    G.dirty = true;
    g->arena.release(S.off, S.bytes);
    S.used = false;
    return NB_OK;
}

}  // namespace nekgb

using namespace nekgb;

extern "C" {

nb_status nb_engine_create(nb_engine **out, size_t arena_bytes, void *cuda_stream) {
    try {
        if (!out) return fail(NB_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (arena_bytes < ((size_t)1 << 20)) return fail(NB_ERR_ARG, "arena must be at least 1 MiB");
        nb_engine *g = new nb_engine();
        g->stream = (cudaStream_t)cuda_stream;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = dev_alloc((void **)&g->arena.base, arena_bytes);
        if (e != cudaSuccess) { delete g; return cuda_fail(e, "engine: arena"); }
        g->arena.cap = arena_bytes;
        g->arena.free_[0] = arena_bytes & ~(size_t)255;
        if ((e = dev_alloc((void **)&g->d_desc, sizeof(ProbDesc) * kEngMaxSlots)) != cudaSuccess ||
            (e = cudaMallocHost((void **)&g->h_desc, sizeof(ProbDesc) * kEngMaxSlots)) != cudaSuccess) {
            cudaFree(g->arena.base);
            if (g->d_desc) cudaFree(g->d_desc);
            delete g;
            return cuda_fail(e, "engine: descriptors");
        }
        memset(g->h_desc, 0, sizeof(ProbDesc) * kEngMaxSlots);
        for (int k = 0; k < kEngMaxSlots; k++) g->h_desc[k].sc.done = 1;
        e = cudaMemcpyAsync(g->d_desc, g->h_desc, sizeof(ProbDesc) * kEngMaxSlots, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            cudaFree(g->arena.base); cudaFree(g->d_desc); cudaFreeHost(g->h_desc);
            delete g;
            return cuda_fail(e, "engine: init");
        }
        *out = g;
        return NB_OK;
    } catch (...) {
        return fail(NB_ERR_OOM, "engine: host allocation failed");
    }
}

nb_status nb_engine_destroy(nb_engine *g) {
    if (!g) return NB_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    for (int n = 0; n <= kMaxN; n++) {
        NGroup &G = g->groups[n];
        if (G.d_ax) cudaFree(G.d_ax);
        if (G.d_ds) cudaFree(G.d_ds);
        if (G.d_cnt) cudaFree(G.d_cnt);
    }
    cudaFree(g->arena.base);
    cudaFree(g->d_desc);
    cudaFreeHost(g->h_desc);
    delete g;
    return NB_OK;
}

nb_status nb_engine_footprint(nb_box mesh, int n, size_t *bytes) {
    if (!bytes) return fail(NB_ERR_ARG, "NULL argument");
    if (n < 2 || n > kMaxN || mesh.ex < 1 || mesh.ey < 1 || mesh.ez < 1) return fail(NB_ERR_ARG, "bad mesh");
    size_t parts[3];
    *bytes = desc_footprint(make_mesh(mesh, n), 4, parts);
    return NB_OK;
}

nb_status nb_engine_submit(nb_engine *g, const nb_request *req, const double *f_dev, int *id_out) {
    try {
        if (!g || !req || !f_dev || !id_out) return fail(NB_ERR_ARG, "NULL argument");
        if (req->n < 2 || req->n > kMaxN || req->mesh.ex < 1 || req->mesh.ey < 1 || req->mesh.ez < 1)
            return fail(NB_ERR_ARG, "bad mesh");
        if (req->maxit < 0) return fail(NB_ERR_ARG, "maxit must be >= 0");
        if (((uintptr_t)f_dev & 7u)) return fail(NB_ERR_ARG, "f must be 8-byte aligned");
        nb_status s = autotune(g, req->n);
        if (s != NB_OK) return s;
        return engine_submit_internal(g, req->mesh, req->n, req->amp, req->s, req->tol, req->maxit, f_dev,
                                      g->groups[req->n].te, id_out);
    } catch (...) {
        return fail(NB_ERR_OOM, "engine: host allocation failed");
    }
}

nb_status nb_engine_submit_unique(nb_engine *g, const nb_request *req, const double *fu_dev, int *id_out) {
    try {
        if (!g || !req || !fu_dev || !id_out) return fail(NB_ERR_ARG, "NULL argument");
        if (req->n < 2 || req->n > kMaxN || req->mesh.ex < 1 || req->mesh.ey < 1 || req->mesh.ez < 1)
            return fail(NB_ERR_ARG, "bad mesh");
        if (req->maxit < 0) return fail(NB_ERR_ARG, "maxit must be >= 0");
        if (((uintptr_t)fu_dev & 7u)) return fail(NB_ERR_ARG, "f must be 8-byte aligned");
        nb_status s = autotune(g, req->n);
        if (s != NB_OK) return s;
        return engine_submit_internal(g, req->mesh, req->n, req->amp, req->s, req->tol, req->maxit, fu_dev,
                                      g->groups[req->n].te, id_out, true);
    } catch (...) {
        return fail(NB_ERR_OOM, "engine: host allocation failed");
    }
}

nb_status nb_engine_step(nb_engine *g, int iters) {
    try {
        if (!g) return fail(NB_ERR_ARG, "NULL engine");
        return engine_step_internal(g, iters);
    } catch (...) {
        return fail(NB_ERR_OOM, "engine: host allocation failed");
    }
}

nb_status nb_engine_poll(nb_engine *g, int id, int *done, int *iters, double *relres, int *status) {
    if (!g || id < 0 || id >= kEngMaxSlots || !g->slots[id].used) return fail(NB_ERR_ARG, "unknown request id");
    const CgScalars &sc = g->h_desc[id].sc;
    if (done) *done = sc.done;
    if (iters) *iters = sc.it;
    if (relres) *relres = sc.fnorm2 > 0.0 ? sqrt(sc.rho) / sqrt(sc.fnorm2) : 0.0;
    if (status) {
        nb_status st = NB_OK;
        if (sc.status == (int)NB_ERR_BREAKDOWN) st = NB_ERR_BREAKDOWN;
        else if (sc.done && sc.tol > 0.0 && sc.rho != 0.0 && !(sqrt(sc.rho) / sqrt(sc.fnorm2) <= sc.tol))
            st = NB_ERR_NOT_CONVERGED;
        *status = (int)st;
    }
    return NB_OK;
}

nb_status nb_engine_retire(nb_engine *g, int id, double *x_dev) {
    try {
        if (!g) return fail(NB_ERR_ARG, "NULL engine");
        if (x_dev && ((uintptr_t)x_dev & 7u)) return fail(NB_ERR_ARG, "x must be 8-byte aligned");
        return engine_retire_internal(g, id, x_dev);
    } catch (...) {
        return fail(NB_ERR_OOM, "engine: host allocation failed");
    }
}

nb_status nb_engine_stats(const nb_engine *g, size_t *used, size_t *capacity, int *active) {
    if (!g) return fail(NB_ERR_ARG, "NULL engine");
    if (used) *used = g->arena.used;
    if (capacity) *capacity = g->arena.cap;
    if (active) {
        int a = 0;
        for (int k = 0; k < kEngMaxSlots; k++) a += g->slots[k].used ? 1 : 0;
        *active = a;
    }
    return NB_OK;
}

nb_status nb_engine_tuning(const nb_engine *g, int n, int *lines_per_thread, int *elems_per_tile) {
    if (!g || n < 2 || n > kMaxN) return fail(NB_ERR_ARG, "bad argument");
    if (lines_per_thread) *lines_per_thread = g->groups[n].lpt;
    if (elems_per_tile) *elems_per_tile = g->groups[n].te;
    return NB_OK;
}

}  // extern "C"
