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
// * Autotuning: for each (n, precision) the first use times the CG
//   iteration with one or two line tasks per thread (FP64 heads) and 4, 8
//   or 16 elements per tile on a synthetic problem, and caches the choice
//   (NEKGB_TUNE_CACHE file).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ax_df_core.cuh"
#include "ax_f32_core.cuh"
#include "gs_fast.cuh"
#include "gs_nodes.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

constexpr int kEngMaxSlots = 1024;
constexpr int kDsTile = 2048;   // shared nodes per dssum tile (256 threads x 8)
constexpr int kEngThreads = 256;

// Mixed-precision request phases (defect correction, as in mixed.cu).
constexpr int kPhaseInner = 0;   // FP32 inner CG iterating
constexpr int kPhaseOuter = 1;   // FP64 residual step due
constexpr int kPhaseDone = 2;

struct ProbDesc {
    Mesh m;
    float2 *g;                  // gxyz pairs [E][6][n^3]
    double *r, *p, *w, *x;      // CG vectors, local storage (mixed: r, p unused)
    double *partials;           // FP64: ntile_ax + ntile_ds slots; mixed: 2 ntile_ax + ntile_ds
    int ntile_ax, ntile_ds, te;
    int cx, cy, cz;
    int prec;                   // NB_FP64 or NB_MIXED
    // FP64: sc is the CG state.  Mixed: sc holds the outer state (rr =
    // <r,r>_c of the FP64 residual, fnorm2, tol, maxit = inner-iteration
    // budget, it = inner iterations so far, done, status) and si the inner
    // FP32 CG's scalars.
    CgScalars sc;
    CgScalars si;
    int phase, outer, max_outer, pad;
    double inner_tol;
    DsCat dd;                   // shared-node decode of the mesh (by category)
    double *f;                  // mixed: right-hand side (FP64, masked)
    float *g32;                 // mixed: gxyz FP32 [E][6][n^3]
    float *r32, *p32, *w32, *z32;
};

// ---------------------------------------------------------------- kernels
// The FP64 CG head on one tile (elements e0 .. e1-1 of problem P): the
// single-problem head's element loop (ax_df.cu, cg_head_pipelined) over the
// tile's consecutive elements.  The pairs of p are scaled by one power of
// two per problem and iteration, 2^sh with sqrt(<p,p>_c) 2^sh in [1, 2)
// (<p,p>_c carried by eng_assemble), so no element needs an exponent scan;
// the six shared arrays rotate roles between consecutive elements, so the
// next element is staged while the current one's partials are summed: four
// barriers per element.  Returns this thread's share of the tile's <w,p>_c
// (local products at the points off the box faces), an FP64 sum in element
// order, so the tile's partial does not depend on which CTA computed it.
template <int N, int T>
__device__ __forceinline__ double eng_head_tile(const ProbDesc &P, int64_t e0, int64_t e1, double beta,
                                                double xa, const DfEo<N> &D, float2 *sm,
                                                const FaceBits<N, T, df_points_per_thread<N, T>()> &pf) {
    constexpr int N2 = N * N, N3 = N * N * N;
    const int t = threadIdx.x;
    const double pn = P.sc.it == 0 ? P.sc.rr : P.sc.pn2;
    const int ep = (int)((__double_as_longlong(pn) >> 52) & 0x7ff);
    const int sh_in = ep == 0 ? 0 : -((ep - 1023) >> 1);
    const int sh_out = -sh_in;           // the engine's gxyz pairs are unscaled
    float2 *S0 = sm, *S1 = sm + N3, *S2 = sm + 2 * N3, *S3 = sm + 3 * N3, *S4 = sm + 4 * N3, *S5 = sm + 5 * N3;
    const Mesh m = P.m;
    // x += xa p (the owed update), p = r + beta p, X = pairs of p 2^sh
    auto stage = [&](int64_t e, float2 *X) {
        const int64_t eb = e * N3;
        double *p = P.p + eb;
        const double *r = P.r + eb;
        if (xa != 0.0) {
            double *x = P.x + eb;
            for (int q = t; q < N3; q += T) {
                const double pold = p[q];
                __stcs(x + q, fma(xa, pold, __ldcs(x + q)));
                const double v = fma(beta, pold, r[q]);
                p[q] = v;
                X[q] = dfa::split_scaled<true>(v, sh_in);
            }
        } else {
            for (int q = t; q < N3; q += T) {
                const double v = fma(beta, p[q], r[q]);
                p[q] = v;
                X[q] = dfa::split_scaled<true>(v, sh_in);
            }
        }
    };
    double de = 0.0;
    stage(e0, S0);
    __syncthreads();
    for (int64_t e = e0; e < e1; e++) {
        const bool odd = (e - e0) & 1;
        float2 *X = odd ? S1 : S0;
        float2 *F0 = odd ? S0 : S1;
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            float2 *Fd = task < N2 ? F0 : (task < 2 * N2 ? S2 : S3);
            line_eo<N>(X, Fd, base, stride, D.fwd);
        }
        __syncthreads();
        const float2 *g = P.g + e * 6 * N3;
        for (int q = t; q < N3; q += T) {
            const float2 wr = F0[q], ws = S2[q], wt = S3[q];
            const float2 g0 = __ldcs(g + q), g1 = __ldcs(g + N3 + q), g2 = __ldcs(g + 2 * N3 + q);
            const float2 g3 = __ldcs(g + 3 * N3 + q), g4 = __ldcs(g + 4 * N3 + q), g5 = __ldcs(g + 5 * N3 + q);
            dfa::Acc ur = dfa::first(g0.x, g0.y, wr.x, wr.y);
            dfa::fma(ur, g1.x, g1.y, ws.x, ws.y);
            dfa::fma(ur, g2.x, g2.y, wt.x, wt.y);
            dfa::Acc us = dfa::first(g1.x, g1.y, wr.x, wr.y);
            dfa::fma(us, g3.x, g3.y, ws.x, ws.y);
            dfa::fma(us, g4.x, g4.y, wt.x, wt.y);
            dfa::Acc ut = dfa::first(g2.x, g2.y, wr.x, wr.y);
            dfa::fma(ut, g4.x, g4.y, ws.x, ws.y);
            dfa::fma(ut, g5.x, g5.y, wt.x, wt.y);
            F0[q] = dfa::raw(ur);
            S2[q] = dfa::raw(us);
            S3[q] = dfa::raw(ut);
        }
        __syncthreads();
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            const float2 *Fd = task < N2 ? F0 : (task < 2 * N2 ? S2 : S3);
            float2 *Pd = task < N2 ? X : (task < 2 * N2 ? S4 : S5);
            line_eo<N>(Fd, Pd, base, stride, D.bwd);
        }
        // the tile's next element into L2, about one element ahead of its stage
        // (r, p, x) and its contraction (the geometric factors): +7 % on the
        // 256-problem batch.  (The single-problem head measured faster by 1 %
        // with the same hint but moved 31 MB more DRAM traffic per launch and
        // slowed the update kernel that follows by 8 %, so it has none.)
        if (t == 0 && e + 1 < e1) {
            l2_prefetch(P.g + (e + 1) * 6 * N3, sizeof(float2) * 6 * N3);
            l2_prefetch(P.r + (e + 1) * N3, sizeof(double) * N3);
            l2_prefetch(P.p + (e + 1) * N3, sizeof(double) * N3);
            if (xa != 0.0) l2_prefetch(P.x + (e + 1) * N3, sizeof(double) * N3);
        }
        __syncthreads();
        {
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            const unsigned bf = box_faces(ex, ey, ez, m);
            const int64_t eb = e * N3;
            const double *p = P.p + eb;
            double *w = P.w + eb;
#pragma unroll
            for (int kk = 0; kk < df_points_per_thread<N, T>(); kk++) {
                const int q = t + kk * T;
                if (df_points_per_thread<N, T>() * T != N3 && q >= N3) break;
                const float2 sum = dfa::add(dfa::add(X[q], S4[q]), S5[q]);
                double wv = dfa::join_scaled(sum, sh_out);
                if (pf[kk] & bf)
                    wv = 0.0;
                else
                    de = fma(wv, p[q], de);
                w[q] = wv;
            }
        }
        if (e + 1 < e1) stage(e + 1, odd ? S0 : S1);
        __syncthreads();
    }
    return de;
}

// CG head over a list of (slot, tile) work units.
template <int N, int T>
__global__ void __launch_bounds__(T, df_min_blocks<N, T, 48>())
eng_ax_head(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, int *__restrict__ ntiles,
            const __grid_constant__ DfEo<N> D) {
    extern __shared__ float2 sm[];
    __shared__ int s_last;
    __shared__ double red[32];
    FaceBits<N, T, df_points_per_thread<N, T>()> pf;
    pf.init();
    // Tiles after the first come from a counter (ntiles[2]), so that SMs
    // that run slower take fewer; a tile's result does not depend on the CTA
    // that computes it.  Thread 0 takes the next index at the start of a
    // tile into one of two slots (alternating, so that no thread can still be
    // reading a slot when it is written again) and the CTA reads it after the
    // tile's barriers; the last CTA to leave resets the counter for the next
    // launch (ntiles[3] counts them).
    __shared__ int s_next[2];
    const int nt = ntiles[0];
    int par = 0;
    for (int ti = blockIdx.x; ti < nt; ti = s_next[par], par ^= 1) {
        if (threadIdx.x == 0) s_next[par] = (int)gridDim.x + atomicAdd(ntiles + 2, 1);
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.sc.done) {                             // uniform over the CTA
            __syncthreads();                         // s_next[par] is visible to the CTA
            continue;
        }
        const double beta = P.sc.it == 0 ? 0.0 : P.sc.beta;
        const double xa = P.sc.x_alpha;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < P.m.E ? e0 + P.te : P.m.E;
        const double dot = eng_head_tile<N, T>(P, e0, e1, beta, xa, D, sm, pf);
        // <w,p>_c: the problem's last tile sums the tiles' local products
        // in a fixed order and forms alpha
        const double b = block_sum(dot, red);
        if (threadIdx.x == 0) {
            P.partials[tile.y] = b;
            __threadfence();
            s_last = atomicAdd(&P.sc.ticket, 1u) == (unsigned)P.ntile_ax - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double acc = 0.0;
            for (int k = threadIdx.x; k < P.ntile_ax; k += T) acc += __ldcg(P.partials + k);
            const double pap = block_sum(acc, red);
            if (threadIdx.x == 0) {
                P.sc.ticket = 0;
                finalize_alpha(&P.sc, pap);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();   // this CTA's counter increments come before its exit count
        if (atomicAdd(ntiles + 3, 1) == (int)gridDim.x - 1) {
            ntiles[2] = 0;
            ntiles[3] = 0;
        }
    }
}

// Second kernel of an engine CG iteration (as assemble.cu for one
// problem): over the element tiles, r -= alpha w at the element-interior
// points; over the node tiles, each shared node gathers its copies of w in the
// dssum order, updates r once and writes it to every copy.  <r,r>_c is
// summed over unique nodes; the problem's last tile forms rho, beta and the
// convergence decision (MIXED: of the inner FP32 solve, which hands the
// problem to the outer step when it ends).
template <typename T, int N, bool MIXED>
__global__ void __launch_bounds__(kEngThreads, 5)
eng_assemble(ProbDesc *__restrict__ desc, const int2 *__restrict__ ax_tiles, const int2 *__restrict__ ds_tiles,
             const int *__restrict__ cnt) {
    constexpr int N3 = N * N * N;
    constexpr int NI = N > 2 ? N - 2 : 1, NI3 = N > 2 ? NI * NI * NI : 0;
    constexpr int KI = (NI3 + kEngThreads - 1) / kEngThreads;
    __shared__ double red[32];
    __shared__ int s_last;
    int qk[KI > 0 ? KI : 1];   // this thread's element-interior points
#pragma unroll
    for (int k = 0; k < KI; k++) {
        const int qi = threadIdx.x + k * kEngThreads;
        qk[k] = (1 + qi % NI) + N * (1 + (qi / NI) % NI) + N * N * (1 + qi / (NI * NI));
    }
    const int nax = cnt[0], nds = cnt[1];
    for (int ti = blockIdx.x; ti < nax + nds; ti += gridDim.x) {
        const bool el = ti < nax;
        const int2 tile = el ? ax_tiles[ti] : ds_tiles[ti - nax];
        ProbDesc &P = desc[tile.x];
        if (MIXED) {
            if (P.phase != kPhaseInner || P.si.done) continue;
        } else {
            if (P.sc.done) continue;
        }
        CgScalars &S = MIXED ? P.si : P.sc;
        const Mesh m = P.m;
        T *r;
        const T *w;
        if constexpr (MIXED) { r = P.r32; w = P.w32; }
        else { r = P.r; w = P.w; }
        const T alpha = (T)S.alpha;
        const int erb = (int)((__double_as_longlong(S.rr) >> 52) & 0x7ff);
        const int sh = erb == 0 ? 0 : -((erb - 1023) >> 1);
        dfa::SqAcc32 sq;
        dfa::Acc32 acc32;
        auto add_sq = [&](T rn) {
            if constexpr (MIXED) {
                acc32.add_prod(rn, rn);
            } else {
                const float2 v = dfa::split_scaled<true>(rn, sh);
                sq.add_sq(v.x, v.y, 1.f);
            }
        };
        if (el) {   // element-interior points (box-face points stay +0.0, see assemble.cu)
            if constexpr (N > 2) {
                const int64_t e0 = (int64_t)tile.y * P.te;
                const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
                for (int64_t e = e0; e < e1; e++) {
                    const int64_t base = e * N3;
#pragma unroll
                    for (int k = 0; k < KI; k++) {
                        if (KI * kEngThreads != NI3 && threadIdx.x + k * kEngThreads >= NI3) break;
                        const int64_t q = base + qk[k];
                        const T rn = fma(-alpha, __ldcs(w + q), r[q]);
                        r[q] = rn;
                        add_sq(rn);
                    }
                }
            }
        } else {
            const int total = P.cx + P.cy + P.cz;
            const int q0 = tile.y * kDsTile;
            const int q1 = q0 + kDsTile < total ? q0 + kDsTile : total;
            for (int q = q0 + threadIdx.x; q < q1; q += kEngThreads) {
                int64_t idx[8];
                const int c = cat_copies<N>(q, P.dd, idx);
                T sum;
                if (c == 2) {
                    sum = plus_zero(__ldcs(w + idx[0])) + __ldcs(w + idx[1]);
                } else if (c == 4) {
                    T a[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) a[k] = __ldcs(w + idx[k]);
                    sum = plus_zero(a[0]);
#pragma unroll
                    for (int k = 1; k < 4; k++) sum = sum + a[k];
                } else {
                    T a[8];
#pragma unroll
                    for (int k = 0; k < 8; k++) a[k] = __ldcs(w + idx[k]);
                    sum = plus_zero(a[0]);
#pragma unroll
                    for (int k = 1; k < 8; k++) sum = sum + a[k];
                }
                const T rn = fma(-alpha, sum, r[idx[0]]);
                for (int k = 0; k < c; k++) r[idx[k]] = rn;
                add_sq(rn);
            }
        }
        double v;
        if constexpr (MIXED) v = acc32.value();
        else v = sq.value() * __longlong_as_double((long long)(1023 - 2 * sh) << 52);
        const double b = block_sum(v, red);
        if (threadIdx.x == 0) {
            P.partials[el ? tile.y : P.ntile_ax + tile.y] = b;
            __threadfence();
            s_last = atomicAdd(&S.ticket, 1u) == (unsigned)(P.ntile_ax + P.ntile_ds) - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double a2 = 0.0;
            const int cntp = P.ntile_ax + P.ntile_ds;
            for (int k = threadIdx.x; k < cntp; k += kEngThreads) a2 += __ldcg(P.partials + k);
            const double rho = block_sum(a2, red);
            if (threadIdx.x == 0) {
                S.ticket = 0;
                // <p,p>_c of the next search direction: r' is orthogonal to
                // p, so <p',p'>_c = rho' + beta^2 <p,p>_c (p_0 = r_0); the
                // FP64 head takes its pair scale from it
                const double pprev = S.it == 0 ? S.rho : S.pn2;
                S.rr = rho;
                S.rho_old = S.rho;
                S.rho = rho;
                S.beta = rho / S.rho_old;
                S.pn2 = fma(S.beta * S.beta, pprev, rho);
                const int it = S.it + 1;
                S.it = it;
                if (MIXED) {
                    P.sc.it += 1;
                    const bool conv = sqrt(rho) / sqrt(S.fnorm2) <= S.tol;
                    if (rho == 0.0 || conv || it >= S.maxit) {
                        S.done = 1;
                        P.phase = kPhaseOuter;
                    }
                } else {
                    const bool conv = S.tol > 0.0 && sqrt(rho) / sqrt(S.fnorm2) <= S.tol;
                    if (rho == 0.0 || conv || it >= S.maxit) S.done = 1;
                }
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
        P.sc.rr = rho;
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
__global__ void eng_scatter_mask(ProbDesc *__restrict__ desc, int slot, const double *__restrict__ fu,
                                 double *__restrict__ dst) {
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
        dst[q] = on_box_face(i, j, k, ex, ey, ez, m) ? 0.0 : fu[gx + m.NX * (gy + m.NY * gz)];
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

// ---------------------------------------------------------------- mixed
// Mixed-precision requests: defect correction with an FP32 inner CG, as in
// mixed.cu, driven per problem on the device.  Each engine step first runs
// the outer pass for the problems whose inner solve ended (x += d, the FP64
// residual r = f - A x with the FP64-accurate operator, the convergence
// test and the start of the next inner solve), then the inner iterations.
// A problem's phase decides which kernels touch it; every decision is taken
// by the problem's own last tile, so results stay independent of the mix.

// Inner CG head over (slot, tile) work units: z += xa p, p = r + beta p,
// w = ax_e(p) in FP32, box faces zeroed, local products w p per tile.
template <int N, int T>
__global__ void __launch_bounds__(T)
eng_m_head(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles,
           const __grid_constant__ F32Mat<N> D) {
    constexpr int N3 = N * N * N;
    extern __shared__ __align__(16) float smf[];
    __shared__ double red[32];
    __shared__ int s_last;
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.phase != kPhaseInner || P.si.done) continue;     // uniform over the CTA
        const float beta = P.si.it == 0 ? 0.f : (float)P.si.beta;
        const float xa = (float)P.si.x_alpha;
        const Mesh m = P.m;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
        dfa::Acc32 dot;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t eb = e * N3;
            F32ElemIO io;
            io.u = nullptr;
            io.r = P.r32 + eb;
            io.p = P.p32 + eb;
            io.x = P.z32 + eb;
            io.w = P.w32 + eb;
            io.g = P.g32 + e * 6 * N3;
            if (threadIdx.x == 0 && e + 1 < e1) {   // the next element into L2 (see eng_head_tile)
                l2_prefetch(P.g32 + (e + 1) * 6 * N3, sizeof(float) * 6 * N3);
                l2_prefetch(P.r32 + (e + 1) * N3, sizeof(float) * N3);
                l2_prefetch(P.p32 + (e + 1) * N3, sizeof(float) * N3);
                if (xa != 0.f) l2_prefetch(P.z32 + (e + 1) * N3, sizeof(float) * N3);
            }
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            f32_element<N, 1, T>(io, beta, xa, ex, ey, ez, m, D, smf, dot);
        }
        // <w,p>_c: the problem's last tile forms alpha (an inner breakdown
        // hands the problem back to the outer step)
        const double b = block_sum(dot.value(), red);
        if (threadIdx.x == 0) {
            P.partials[tile.y] = b;
            __threadfence();
            s_last = atomicAdd(&P.si.ticket, 1u) == (unsigned)P.ntile_ax - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double acc = 0.0;
            for (int k = threadIdx.x; k < P.ntile_ax; k += T) acc += __ldcg(P.partials + k);
            const double pap = block_sum(acc, red);
            if (threadIdx.x == 0) {
                P.si.ticket = 0;
                finalize_alpha(&P.si, pap);
                if (P.si.done) P.phase = kPhaseOuter;
            }
        }
        __syncthreads();
    }
}

// The inner head with bulk-copy staging (f32_element_staged): each CTA walks
// its work items -- the elements of its active tiles, in order -- and
// while it computes one, the copy engine brings the next one's r, p, z
// slabs into the other stage, across tile and problem boundaries (the
// geometric factors go straight to registers).  A tile's last element closes the tile's <w,p> partial; a
// problem's last tile forms alpha.  A copy that does not complete within
// ~1 s ends the CTA after draining its copies and marks the problem it was
// on with NB_ERR_TIMEOUT.  Even n <= 10 (16-byte aligned slabs).
template <int N, int T>
__global__ void __launch_bounds__(T, f32_staged_min_blocks<N>())
eng_m_head_staged(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles,
                  const __grid_constant__ F32Mat<N> D) {
    constexpr int N3 = N * N * N;
    constexpr int STAGE = f32_stage_floats<N, 1>();
    extern __shared__ __align__(16) float smf[];
    __shared__ double red[32];
    __shared__ int s_last;
    __shared__ __align__(8) uint64_t bars[2];
    const int t = threadIdx.x;
    const int nt = *ntiles;
    struct Item {
        int ti;
        int64_t e, e1;
    };
    // the first active tile at ti or later (stride gridDim.x); the flags of
    // a tile this CTA has not processed yet cannot change meanwhile (only a
    // problem's last tile changes them)
    auto first_from = [&](int ti, Item &it) -> bool {
        for (; ti < nt; ti += gridDim.x) {
            const int2 tile = tiles[ti];
            const ProbDesc &P = desc[tile.x];
            if (P.phase != kPhaseInner || P.si.done) continue;
            it.ti = ti;
            it.e = (int64_t)tile.y * P.te;
            it.e1 = it.e + P.te < P.m.E ? it.e + P.te : P.m.E;
            return true;
        }
        return false;
    };
    auto advance = [&](Item &it) -> bool {
        if (it.e + 1 < it.e1) {
            it.e++;
            return true;
        }
        return first_from(it.ti + (int)gridDim.x, it);
    };
    Item cur;
    if (!first_from(blockIdx.x, cur)) return;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t pol = t == 0 ? l2_evict_first_policy() : 0ull;
    auto issue = [&](const Item &it, int s) {   // thread 0
        const ProbDesc &P = desc[tiles[it.ti].x];
        const bool wx = (float)P.si.x_alpha != 0.f;
        float *st = smf + s * STAGE;
        mbar_expect_tx(&bars[s], 4u * (wx ? 3 : 2) * N3);
        bulk_g2s(st, P.r32 + it.e * N3, 4u * N3, &bars[s]);
        bulk_g2s(st + N3, P.p32 + it.e * N3, 4u * N3, &bars[s]);
        if (wx) bulk_g2s_hint(st + 2 * N3, P.z32 + it.e * N3, 4u * N3, &bars[s], pol);
    };
    int issued[2] = {1, 0}, waited[2] = {0, 0};
    if (t == 0) issue(cur, 0);
    unsigned pf[f32_points_per_thread<N, T>()];
    f32_point_masks<N, T>(pf);
    float gv[f32_points_per_thread<N, T>()][6];
    f32_load_factors<N, T>(desc[tiles[cur.ti].x].g32 + cur.e * 6 * N3, gv);
    dfa::Acc32 dot;
    bool ok = true;
    for (int i = 0;; i++) {
        const int s = i & 1;
        Item nxt = cur;
        const bool more = advance(nxt);
        if (more) {
            if (t == 0) issue(nxt, s ^ 1);
            issued[s ^ 1]++;
        }
        ok = __syncthreads_and(mbar_wait(&bars[s], waited[s] & 1)) != 0;
        if (!ok) break;
        waited[s]++;
        const int2 tile = tiles[cur.ti];
        ProbDesc &P = desc[tile.x];
        const float beta = P.si.it == 0 ? 0.f : (float)P.si.beta;
        const float xa = (float)P.si.x_alpha;
        F32StagedOut o;
        o.p = P.p32 + cur.e * N3;
        o.x = P.z32 + cur.e * N3;
        o.w = P.w32 + cur.e * N3;
        int ex, ey, ez;
        element_coords(cur.e, P.m, ex, ey, ez);
        f32_element_staged<N, 1, T>(smf + s * STAGE, smf + 2 * STAGE, gv,
                                    more ? desc[tiles[nxt.ti].x].g32 + nxt.e * 6 * N3 : nullptr, o, beta, xa, ex,
                                    ey, ez, P.m, D, dot, pf);
        if (cur.e + 1 == cur.e1) {   // the tile is complete
            const double b = block_sum(dot.value(), red);
            dot = dfa::Acc32();
            if (t == 0) {
                P.partials[tile.y] = b;
                __threadfence();
                s_last = atomicAdd(&P.si.ticket, 1u) == (unsigned)P.ntile_ax - 1;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                double acc = 0.0;
                for (int k = t; k < P.ntile_ax; k += T) acc += __ldcg(P.partials + k);
                const double pap = block_sum(acc, red);
                if (t == 0) {
                    P.si.ticket = 0;
                    finalize_alpha(&P.si, pap);
                    if (P.si.done) P.phase = kPhaseOuter;
                }
            }
            __syncthreads();
        }
        if (!more) break;
        cur = nxt;
    }
    if (!ok && t == 0) {   // drain the copies in flight, then report on the current problem
        for (int s = 0; s < 2; s++)
            if (issued[s] > waited[s]) mbar_wait(&bars[s], waited[s] & 1);
        ProbDesc &P = desc[tiles[cur.ti].x];
        P.sc.status = (int)NB_ERR_TIMEOUT;
        P.sc.done = 1;
        P.phase = kPhaseDone;
    }
}

// Outer step: shared-node sums of the FP64 w = A x over (slot, node tile)
// work units (ascending element order, as dssum).  Skipped on the first
// pass (x = 0, so A x = 0).
template <int N>
__global__ void __launch_bounds__(kEngThreads)
eng_outer_dssum(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles) {
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.phase != kPhaseOuter || P.outer == 0) continue;
        const int total = P.cx + P.cy + P.cz;
        double *w = P.w;
        const int q0 = tile.y * kDsTile;
        const int q1 = q0 + kDsTile < total ? q0 + kDsTile : total;
        for (int q = q0 + threadIdx.x; q < q1; q += kEngThreads) {
            int64_t idx[8];
            const int c = cat_copies<N>(q, P.dd, idx);
            double sum;
            if (c == 2) {
                sum = plus_zero(w[idx[0]]) + w[idx[1]];
            } else if (c == 4) {
                double a[4];
#pragma unroll
                for (int k = 0; k < 4; k++) a[k] = w[idx[k]];
                sum = plus_zero(a[0]);
#pragma unroll
                for (int k = 1; k < 4; k++) sum = sum + a[k];
            } else {
                double a[8];
#pragma unroll
                for (int k = 0; k < 8; k++) a[k] = w[idx[k]];
                sum = plus_zero(a[0]);
#pragma unroll
                for (int k = 1; k < 8; k++) sum = sum + a[k];
            }
            for (int k = 0; k < c; k++) w[idx[k]] = sum;
        }
    }
}

// Outer step, part 1: x += d, with d = z + x_alpha p (the inner solve's
// owed update), in FP64.  Skipped on the first pass (x = 0, no inner solve).
template <int N>
__global__ void __launch_bounds__(kEngThreads)
eng_m_outer_x(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles) {
    constexpr int N3 = N * N * N;
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const ProbDesc &P = desc[tile.x];
        if (P.phase != kPhaseOuter || P.outer == 0) continue;
        const float xa = (float)P.si.x_alpha;
        const int64_t q0 = (int64_t)tile.y * P.te * N3;
        const int64_t q1 = (int64_t)(tile.y + 1) * P.te * N3 < P.m.npts ? (int64_t)(tile.y + 1) * P.te * N3
                                                                          : P.m.npts;
        for (int64_t q = q0 + threadIdx.x; q < q1; q += kEngThreads) {
            const float d = fmaf(xa, P.p32[q], P.z32[q]);
            P.x[q] += (double)d;
        }
    }
}

// Outer step, part 2: w = ax_e(x) with the FP64-accurate (double-float)
// element operator.  Skipped on the first pass.
template <int N, int T>
__global__ void __launch_bounds__(T)
eng_m_outer_ax(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles,
               const __grid_constant__ DfEo<N> D) {
    constexpr int N3 = N * N * N;
    extern __shared__ float2 sm[];
    __shared__ int s_emax;
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const ProbDesc &P = desc[tile.x];
        if (P.phase != kPhaseOuter || P.outer == 0) continue;
        const Mesh m = P.m;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
        double dot = 0.0;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t eb = e * N3;
            DfElemIO io;
            io.u = P.x + eb;
            io.r = nullptr;
            io.p = nullptr;
            io.x = nullptr;
            io.minv = nullptr;
            io.w = P.w + eb;
            io.g = P.g + e * 6 * N3;
            df_element<N, 0, true, T>(io, 0.0, 0.0, false, 1023, m, 0, 0, 0, D, sm, &s_emax, dot);
        }
    }
}

// Outer step, part 3: r = mask(f - w) (w = A x after dssum; A x = 0 on the
// first pass), rr = <r,r>_c in FP64, and the inner right-hand side
// r32 = fl32(r) with p32 = z32 = 0 and rho32 = <r32,r32>_c.  The problem's
// last tile decides: converged (or out of budget) -> done; otherwise the
// next inner solve starts.
template <int N>
__global__ void __launch_bounds__(kEngThreads)
eng_m_outer_resid(ProbDesc *__restrict__ desc, const int2 *__restrict__ tiles, const int *__restrict__ ntiles) {
    constexpr int N3 = N * N * N;
    __shared__ double red[32];
    __shared__ int s_last;
    const int nt = *ntiles;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        ProbDesc &P = desc[tile.x];
        if (P.phase != kPhaseOuter) continue;
        const Mesh m = P.m;
        const bool first = P.outer == 0;
        const int64_t e0 = (int64_t)tile.y * P.te;
        const int64_t e1 = e0 + P.te < m.E ? e0 + P.te : m.E;
        double acc = 0.0;
        dfa::Acc32 acc32;
        for (int64_t e = e0; e < e1; e++) {
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            const int64_t eb = e * N3;
            for (int q = threadIdx.x; q < N3; q += kEngThreads) {
                const int i = q % N, j = (q / N) % N, k = q / (N * N);
                double rv = 0.0;
                if (!on_box_face(i, j, k, ex, ey, ez, m)) rv = first ? P.f[eb + q] : P.f[eb + q] - P.w[eb + q];
                const int lg = log2_mult(i, j, k, ex, ey, ez, m);
                acc = fma(scale_down_pow2(rv, lg), rv, acc);
                const float r32 = __double2float_rn(rv);
                P.r32[eb + q] = r32;
                P.p32[eb + q] = 0.f;
                P.z32[eb + q] = 0.f;
                acc32.add_prod(r32 * __uint_as_float((unsigned)(127 - lg) << 23), r32);
            }
        }
        const double b = block_sum(acc, red);
        const double b32 = block_sum(acc32.value(), red);
        if (threadIdx.x == 0) {
            P.partials[tile.y] = b;
            P.partials[P.ntile_ax + P.ntile_ds + tile.y] = b32;
            __threadfence();
            const unsigned t = atomicAdd(&P.sc.ticket, 1u);
            s_last = (t == (unsigned)P.ntile_ax - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double a2 = 0.0, a3 = 0.0;
            for (int k = threadIdx.x; k < P.ntile_ax; k += kEngThreads) {
                a2 += __ldcg(P.partials + k);
                a3 += __ldcg(P.partials + P.ntile_ax + P.ntile_ds + k);
            }
            const double rr = block_sum(a2, red);
            const double rho32 = block_sum(a3, red);
            if (threadIdx.x == 0) {
                P.sc.ticket = 0;
                P.sc.rr = rr;
                P.sc.rho = rr;
                if (first) P.sc.fnorm2 = rr;
                const bool conv = rr == 0.0 || (P.sc.tol > 0.0 && sqrt(rr) / sqrt(P.sc.fnorm2) <= P.sc.tol);
                if (conv || P.outer >= P.max_outer || P.sc.it >= P.sc.maxit) {
                    P.phase = kPhaseDone;
                    P.sc.done = 1;
                } else {
                    CgScalars &si = P.si;
                    si.rho = rho32;
                    si.rr = rho32;
                    si.rho_old = 1.0;
                    si.fnorm2 = rho32;
                    si.beta = 0.0;
                    si.alpha = 0.0;
                    si.x_alpha = 0.0;
                    si.it = 0;
                    si.status = 0;
                    si.tol = P.inner_tol;
                    si.maxit = P.sc.maxit - P.sc.it;
                    si.done = rho32 == 0.0 ? 1 : 0;
                    P.outer += 1;
                    P.phase = si.done ? kPhaseOuter : kPhaseInner;
                }
            }
        }
        __syncthreads();
    }
}

// FP32 geometric factors of a mixed request from its pairs (h + l): h.
__global__ void eng_pairs_to_f32(const float2 *__restrict__ g, float *__restrict__ g32, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        g32[q] = g[q].x;
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
    int prec = 0;
    size_t off = 0, bytes = 0;
    double t_submit = 0.0;
};

struct NGroup {
    int lpt = 0, te = 0;                 // tuned (0: not yet)
    int2 *d_ax = nullptr, *d_ds = nullptr;
    int *d_cnt = nullptr;                // [0] = ax tiles, [1] = dssum tiles, [2] [3] the FP64 head's tile counter
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
    nekgb::NGroup groups[nekgb::kMaxN + 1];    // FP64 requests, per n
    nekgb::NGroup mgroups[nekgb::kMaxN + 1];   // mixed-precision requests, per n
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_key = 0;
    int graph_chunk = 0;
    int sms = 1;
    bool f32_plain = false;   // FP32 heads without bulk staging (NEKGB_F32_STAGED=0)
};

namespace nekgb {

// Arena bytes of one request.  FP64: gxyz pairs, four CG vectors (r, p, w,
// x) and the tile partials.  Mixed: gxyz pairs and FP32 gxyz, three FP64
// vectors (f, w, x), four FP32 vectors (r, p, w, z) and the partials.
static size_t desc_footprint(const Mesh &m, int prec, size_t *parts) {
    const int64_t n3 = (int64_t)m.n * m.n * m.n;
    int cx, cy, cz;
    shared_counts(m, cx, cy, cz);
    const int64_t ntax = (m.E + 3) / 4;   // partial slots for the smallest tile (4 elements)
    const int64_t total = (int64_t)cx + cy + cz;
    const int64_t ntds = total > 0 ? (total + kDsTile - 1) / kDsTile : 1;
    parts[0] = Arena::align(sizeof(float2) * 6 * n3 * m.E);          // gxyz pairs
    parts[1] = Arena::align(sizeof(double) * m.npts);                 // each FP64 vector
    parts[2] = Arena::align(sizeof(double) * (2 * ntax + ntds + 1));  // partials
    parts[3] = Arena::align(sizeof(float) * 6 * n3 * m.E);            // FP32 gxyz
    parts[4] = Arena::align(sizeof(float) * m.npts);                  // each FP32 vector
    if (prec == NB_MIXED) return parts[0] + 3 * parts[1] + parts[2] + parts[3] + 4 * parts[4];
    return parts[0] + 4 * parts[1] + parts[2];
}

static Mesh make_mesh(nb_box b, int n) { return make_box_mesh(b.ex, b.ey, b.ez, n); }

// ---- kernel dispatch over (N, LPT)
template <int N, int LPT>
static nb_status head_launch(nb_engine *g, const NGroup &G) {
    constexpr int T = df_threads_lpt(N, LPT);
    const size_t smem = sizeof(float2) * 6 * N * N * N;
    {
        const nb_status s = set_smem(eng_ax_head<N, T>, smem);
        if (s != NB_OK) return s;
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
    eng_assemble<double, N, false><<<g->sms * 5, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_ds, G.d_cnt);
    NB_LAUNCH_CHECK("eng_assemble");
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

// ---- mixed-precision groups
template <int N>
static nb_status mixed_inner_iteration(nb_engine *g, const NGroup &G) {
    constexpr int T = ax_f32_threads(N);
    if constexpr (f32_staged_ok<N>() && N == 10) {   // measured faster in batches at n = 10 only
        if (!g->f32_plain) {
            const size_t ssm = sizeof(float) * f32_staged_smem_floats<N, 1>();
            {
                const nb_status s = set_smem(eng_m_head_staged<N, T>, ssm);
                if (s != NB_OK) return s;
            }
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_m_head_staged<N, T>, T, ssm);
            if (occ < 1) occ = 1;
            F32Mat<N> D;
            for (int q = 0; q < N * N; q++) D.d[q] = (float)G.D[q];
            eng_m_head_staged<N, T><<<g->sms * occ, T, ssm, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt, D);
            NB_LAUNCH_CHECK("eng_m_head_staged");
            eng_assemble<float, N, true><<<g->sms * 5, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_ds,
                                                                                  G.d_cnt);
            NB_LAUNCH_CHECK("eng_assemble<mixed>");
            return NB_OK;
        }
    }
    const size_t smem = sizeof(float) * f32_smem_floats(N);
    {
        const nb_status s = set_smem(eng_m_head<N, T>, smem);
        if (s != NB_OK) return s;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_m_head<N, T>, T, smem);
    if (occ < 1) occ = 1;
    F32Mat<N> D;
    for (int q = 0; q < N * N; q++) D.d[q] = (float)G.D[q];
    eng_m_head<N, T><<<g->sms * occ, T, smem, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt, D);
    NB_LAUNCH_CHECK("eng_m_head");
    eng_assemble<float, N, true><<<g->sms * 5, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_ds, G.d_cnt);
    NB_LAUNCH_CHECK("eng_assemble<mixed>");
    return NB_OK;
}

template <int N>
static nb_status mixed_outer_pass(nb_engine *g, const NGroup &G) {
    constexpr int T = ax_df_threads(N);
    const size_t smem = sizeof(float2) * 6 * N * N * N;
    {
        const nb_status s = set_smem(eng_m_outer_ax<N, T>, smem);
        if (s != NB_OK) return s;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_m_outer_ax<N, T>, T, smem);
    if (occ < 1) occ = 1;
    DfEo<N> D;
    eo_consts<N>(G.D, false, D.fwd);
    eo_consts<N>(G.D, true, D.bwd);
    eng_m_outer_x<N><<<g->sms * 4, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt);
    NB_LAUNCH_CHECK("eng_m_outer_x");
    eng_m_outer_ax<N, T><<<g->sms * occ, T, smem, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt, D);
    NB_LAUNCH_CHECK("eng_m_outer_ax");
    eng_outer_dssum<N><<<g->sms * 8, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ds, G.d_cnt + 1);
    NB_LAUNCH_CHECK("eng_outer_dssum");
    eng_m_outer_resid<N><<<g->sms * 4, kEngThreads, 0, g->stream>>>(g->d_desc, G.d_ax, G.d_cnt);
    NB_LAUNCH_CHECK("eng_m_outer_resid");
    return NB_OK;
}

static nb_status dispatch_mixed(nb_engine *g, int n, bool outer) {
    const NGroup &G = g->mgroups[n];
    switch (n) {
#define NB_CASE(NN) \
    case NN: return outer ? mixed_outer_pass<NN>(g, G) : mixed_inner_iteration<NN>(g, G);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
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
                                 bool f_unique = false, int prec = NB_FP64, double inner_tol = 0.0);
nb_status engine_retire_internal(nb_engine *g, int id, double *x);
nb_status engine_step_internal(nb_engine *g, int iters);

// Time the CG iteration of a synthetic problem for each candidate (lines
// per thread, elements per tile): the median of five 24-iteration runs.
// The problem is a cube of about 128 elements per SM, so that even the
// largest tiles give every resident CTA at least two (a smaller problem
// leaves CTAs idle and favours the smallest tiles, whatever a large batch
// would want).  The default layout (one line per thread, 8 elements per
// tile) is kept unless a candidate is at least 2 % faster, so that run-to-
// run noise does not flip the choice; an arena without room for the problem
// keeps the defaults.
static nb_status autotune(nb_engine *g, int n, int prec) {
    const bool mixed = prec == NB_MIXED;
    NGroup &G = mixed ? g->mgroups[n] : g->groups[n];
    if (G.lpt) return NB_OK;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char key[512];
    snprintf(key, sizeof key, "n%d_%s_sm%d_%.200s", n, mixed ? "mixed" : "fp64", prop.multiProcessorCount,
             prop.name);
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
    float best = 1e30f, dflt = 1e30f;
    const int dl = !mixed && n >= 13 ? 2 : 1, dt = 8;
    int bl = dl, bt = dt;
    int side = 8;
    while (side * side * side < 128 * prop.multiProcessorCount) side++;
    const nb_box box = {side, side, side};
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
        if (mixed && li == 1) break;              // the FP32 head has one thread layout (lines per thread 1)
        if (!mixed && n >= 13 && lpts[li] == 1) continue;
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
            st = engine_submit_internal(g, box, n, 0.05, s3, 0.0, 1 << 30, f, tes[ti], &id, false, prec);
            if (st == NB_ERR_OOM) {   // no room for the tuning problem: keep the defaults
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                cudaFree(f);
                G.lpt = !mixed && n >= 13 ? 2 : 1;
                G.te = 8;
                return NB_OK;
            }
            if (st != NB_OK) break;
            st = engine_step_internal(g, 8);                       // warm-up (and graph capture)
            float runs[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (int rep = 0; rep < 5 && st == NB_OK; rep++) {     // five 24-iteration runs
                cudaEventRecord(a, g->stream);
                st = engine_step_internal(g, 24);
                cudaEventRecord(b, g->stream);
                cudaEventSynchronize(b);
                cudaEventElapsedTime(&runs[rep], a, b);
            }
            for (int i = 1; i < 5; i++)                             // median
                for (int j = i; j > 0 && runs[j] < runs[j - 1]; j--) {
                    const float tmp = runs[j]; runs[j] = runs[j - 1]; runs[j - 1] = tmp;
                }
            const float ms = runs[2];
            if (lpts[li] == dl && tes[ti] == dt) dflt = ms;
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
    if (dflt < 1e30f && dflt <= 1.02f * best) { bl = dl; bt = dt; }
    G.lpt = bl;
    G.te = bt;
    if (st == NB_OK) tune_store(key, bl, bt);
    return st;
}

static nb_status ensure_group(nb_engine *g, NGroup &G, int n, int64_t max_tiles_ax, int64_t max_tiles_ds) {
    if (!G.d_cnt) {
        double xi[kMaxN], w[kMaxN];
        nb_status s = host_gll(n, xi, w);
        if (s != NB_OK) return s;
        if ((s = host_dmat(n, xi, G.D)) != NB_OK) return s;
        cudaError_t e = dev_alloc((void **)&G.d_cnt, 4 * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "alloc tile counts");
        NB_CUDA(cudaMemsetAsync(G.d_cnt, 0, 4 * sizeof(int), g->stream));
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
    for (int gi = 0; gi < 2 * (kMaxN + 1); gi++) {
        const int n = gi % (kMaxN + 1);
        NGroup &G = gi <= kMaxN ? g->groups[n] : g->mgroups[n];
        if (!G.dirty) continue;
        std::vector<int2> ax, ds;
        for (int slot : G.slots) {
            const ProbDesc &P = g->h_desc[slot];
            for (int j = 0; j < P.ntile_ax; j++) ax.push_back(make_int2(slot, j));
            for (int j = 0; j < P.ntile_ds; j++) ds.push_back(make_int2(slot, j));
        }
        nb_status s = ensure_group(g, G, n, (int64_t)ax.size(), (int64_t)ds.size());
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
                                 bool f_unique, int prec, double inner_tol) {
    const Mesh m = make_mesh(box, n);
    const bool mixed = prec == NB_MIXED;
    size_t parts[5];
    const size_t bytes = desc_footprint(m, prec, parts);
    int slot = -1;
    for (int k = 0; k < kEngMaxSlots; k++)
        if (!g->slots[k].used) { slot = k; break; }
    if (slot < 0) return fail(NB_ERR_OOM, "engine: all request slots are in use");
    size_t off = 0;
    if (!g->arena.alloc(bytes, &off))
        return fail(NB_ERR_OOM, "engine: the request's footprint does not fit in the free arena");
    // ensure the group exists (D, counts) before building the problem
    NGroup &G = mixed ? g->mgroups[n] : g->groups[n];
    nb_status s = ensure_group(g, G, n, 0, 0);
    if (s != NB_OK) { g->arena.release(off, bytes); return s; }
    char *base = g->arena.base + off;
    ProbDesc &P = g->h_desc[slot];
    memset(&P, 0, sizeof P);
    P.m = m;
    P.prec = mixed ? NB_MIXED : NB_FP64;
    P.g = (float2 *)base;
    size_t at = parts[0];
    if (mixed) {
        P.f = (double *)(base + at); at += parts[1];
        P.w = (double *)(base + at); at += parts[1];
        P.x = (double *)(base + at); at += parts[1];
        P.partials = (double *)(base + at); at += parts[2];
        P.g32 = (float *)(base + at); at += parts[3];
        P.r32 = (float *)(base + at); at += parts[4];
        P.p32 = (float *)(base + at); at += parts[4];
        P.w32 = (float *)(base + at); at += parts[4];
        P.z32 = (float *)(base + at); at += parts[4];
        P.inner_tol = inner_tol > 0.0 ? inner_tol : 1e-4;
        P.max_outer = 50;
    } else {
        P.r = (double *)(base + at); at += parts[1];
        P.p = (double *)(base + at); at += parts[1];
        P.w = (double *)(base + at); at += parts[1];
        P.x = (double *)(base + at); at += parts[1];
        P.partials = (double *)(base + at); at += parts[2];
    }
    P.te = te;
    shared_counts(m, P.cx, P.cy, P.cz);
    P.dd = make_ds_cat(m);
    P.ntile_ax = (int)((m.E + te - 1) / te);
    const int64_t total = (int64_t)P.cx + P.cy + P.cz;
    P.ntile_ds = total > 0 ? (int)((total + kDsTile - 1) / kDsTile) : 1;
    P.sc.tol = tol;
    P.sc.maxit = maxit;
    P.sc.done = 1;   // not iterated until set up
    P.si.done = 1;
    P.phase = kPhaseDone;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(g->d_desc + slot, &P, sizeof(ProbDesc), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess) {
        g->arena.release(off, bytes);
        return cuda_fail(e, "engine: descriptor upload");
    }
    int *d_bad = (int *)(P.partials);   // scratch: the partials are rewritten before they are read
    double *rhs = mixed ? P.f : P.r;
    if ((e = cudaMemsetAsync(d_bad, 0, sizeof(int), g->stream)) != cudaSuccess) {
        g->arena.release(off, bytes);
        return cuda_fail(e, "engine: clear geometry flag");
    }
    s = launch_box_geometry_pairs(m, amp, s3, G.D, P.g, d_bad, g->stream);
    if (s == NB_OK && !f_unique &&
        (e = cudaMemcpyAsync(rhs, f, sizeof(double) * m.npts, cudaMemcpyDeviceToDevice, g->stream)) != cudaSuccess)
        s = cuda_fail(e, "engine: copy rhs");
    if (s == NB_OK && f_unique) {
        eng_scatter_mask<<<grid_blocks(m.npts, 256, g->sms * 8), 256, 0, g->stream>>>(g->d_desc, slot, f, rhs);
        if ((e = cudaGetLastError()) != cudaSuccess) s = cuda_fail(e, "eng_scatter_mask");
    }
    if (s == NB_OK && mixed) {
        const int64_t ng = (int64_t)6 * m.n * m.n * m.n * m.E;
        eng_pairs_to_f32<<<grid_blocks(ng, 256, g->sms * 8), 256, 0, g->stream>>>(P.g, P.g32, ng);
        if ((e = cudaGetLastError()) != cudaSuccess) s = cuda_fail(e, "eng_pairs_to_f32");
        if (s == NB_OK && (e = cudaMemsetAsync(P.x, 0, sizeof(double) * m.npts, g->stream)) != cudaSuccess)
            s = cuda_fail(e, "engine: clear x");
    }
    int bad = 0;
    if (s == NB_OK && (e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, g->stream)) != cudaSuccess)
        s = cuda_fail(e, "engine: geometry flag");
    if (s == NB_OK && (e = cudaStreamSynchronize(g->stream)) != cudaSuccess) s = cuda_fail(e, "engine: setup");
    if (s == NB_OK && bad) s = fail(NB_ERR_ARG, "engine: the perturbed map folds (|J| <= 0)");
    if (s == NB_OK && !mixed) s = dispatch_start(g, n, slot, P.ntile_ax);
    if (s == NB_OK && mixed) {
        // the first outer pass (of the next step) forms r = f, <f,f>_c and
        // starts the first inner solve
        P.sc.done = maxit == 0 ? 1 : 0;
        P.phase = maxit == 0 ? kPhaseDone : kPhaseOuter;
        if ((e = cudaMemcpyAsync(g->d_desc + slot, &P, sizeof(ProbDesc), cudaMemcpyHostToDevice, g->stream)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
            s = cuda_fail(e, "engine: descriptor upload");
    }
    if (s != NB_OK) {
        g->arena.release(off, bytes);
        return s;
    }
    g->slots[slot].used = true;
    g->slots[slot].n = n;
    g->slots[slot].prec = P.prec;
    g->slots[slot].off = off;
    g->slots[slot].bytes = bytes;
    G.slots.push_back(slot);
    G.dirty = true;
    *id = slot;
    return NB_OK;
}

// One engine step is a captured graph of `chunk` iterations: first the
// outer pass of every n with mixed requests, then per iteration one CG
// iteration per n of FP64 requests and one inner iteration per n of mixed
// requests.
nb_status engine_step_internal(nb_engine *g, int iters) {
    nb_status s = refresh_tiles(g);
    if (s != NB_OK) return s;
    unsigned long long key = 0;
    for (int n = 2; n <= kMaxN; n++) {
        if (!g->groups[n].slots.empty()) key |= 1ull << n;
        if (!g->mgroups[n].slots.empty()) key |= 1ull << (32 + n);
    }
    if (!key || iters <= 0) return NB_OK;
    const int chunk = 8;
    if (!g->graph || g->graph_key != key || g->graph_chunk != chunk) {
        if (g->graph) {
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
        }
        cudaGraph_t gr = nullptr;
        NB_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        for (int n = 2; n <= kMaxN && s == NB_OK; n++)
            if (key & (1ull << (32 + n))) s = dispatch_mixed(g, n, true);
        for (int k = 0; k < chunk && s == NB_OK; k++)
            for (int n = 2; n <= kMaxN && s == NB_OK; n++) {
                if (key & (1ull << n)) s = dispatch_iteration(g, n);
                if (s == NB_OK && (key & (1ull << (32 + n)))) s = dispatch_mixed(g, n, false);
            }
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
    dead.si.done = 1;
    dead.phase = kPhaseDone;
    NB_CUDA(cudaMemcpyAsync(g->d_desc + id, &dead, sizeof(ProbDesc), cudaMemcpyHostToDevice, g->stream));
    NB_CUDA(cudaStreamSynchronize(g->stream));
    NGroup &G = S.prec == NB_MIXED ? g->mgroups[S.n] : g->groups[S.n];
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
        g->sms = device_sms();
        {
            const char *st = getenv("NEKGB_F32_STAGED");
            g->f32_plain = st && st[0] == '0';
        }
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
    for (int gi = 0; gi < 2 * (kMaxN + 1); gi++) {
        NGroup &G = gi <= kMaxN ? g->groups[gi] : g->mgroups[gi - kMaxN - 1];
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

nb_status nb_engine_footprint(nb_box mesh, int n, nb_precision prec, size_t *bytes) {
    if (!bytes) return fail(NB_ERR_ARG, "NULL argument");
    if (n < 2 || n > kMaxN || mesh.ex < 1 || mesh.ey < 1 || mesh.ez < 1) return fail(NB_ERR_ARG, "bad mesh");
    if (prec != NB_FP64 && prec != NB_MIXED) return fail(NB_ERR_ARG, "unknown precision");
    size_t parts[5];
    *bytes = desc_footprint(make_mesh(mesh, n), (int)prec, parts);
    return NB_OK;
}

nb_status nb_engine_submit(nb_engine *g, const nb_request *req, const double *f_dev, int *id_out) {
    try {
        if (!g || !req || !f_dev || !id_out) return fail(NB_ERR_ARG, "NULL argument");
        if (req->n < 2 || req->n > kMaxN || req->mesh.ex < 1 || req->mesh.ey < 1 || req->mesh.ez < 1)
            return fail(NB_ERR_ARG, "bad mesh");
        if (req->maxit < 0) return fail(NB_ERR_ARG, "maxit must be >= 0");
        if (req->prec != NB_FP64 && req->prec != NB_MIXED) return fail(NB_ERR_ARG, "unknown precision");
        if (((uintptr_t)f_dev & 7u)) return fail(NB_ERR_ARG, "f must be 8-byte aligned");
        nb_status s = autotune(g, req->n, (int)req->prec);
        if (s != NB_OK) return s;
        const int te = (req->prec == NB_MIXED ? g->mgroups : g->groups)[req->n].te;
        return engine_submit_internal(g, req->mesh, req->n, req->amp, req->s, req->tol, req->maxit, f_dev, te,
                                      id_out, false, (int)req->prec, req->inner_tol);
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
        if (req->prec != NB_FP64 && req->prec != NB_MIXED) return fail(NB_ERR_ARG, "unknown precision");
        if (((uintptr_t)fu_dev & 7u)) return fail(NB_ERR_ARG, "f must be 8-byte aligned");
        nb_status s = autotune(g, req->n, (int)req->prec);
        if (s != NB_OK) return s;
        const int te = (req->prec == NB_MIXED ? g->mgroups : g->groups)[req->n].te;
        return engine_submit_internal(g, req->mesh, req->n, req->amp, req->s, req->tol, req->maxit, fu_dev, te,
                                      id_out, true, (int)req->prec, req->inner_tol);
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
    if (relres) *relres = sc.fnorm2 > 0.0 ? sqrt(sc.rr) / sqrt(sc.fnorm2) : 0.0;
    if (status) {
        nb_status st = NB_OK;
        if (sc.status == (int)NB_ERR_BREAKDOWN) st = NB_ERR_BREAKDOWN;
        else if (sc.done && sc.tol > 0.0 && sc.rr != 0.0 && !(sqrt(sc.rr) / sqrt(sc.fnorm2) <= sc.tol))
            st = NB_ERR_NOT_CONVERGED;
        *status = (int)st;
    }
    return NB_OK;
}

nb_status nb_engine_request_info(nb_engine *g, int id, int *prec, int *outer) {
    if (!g || id < 0 || id >= kEngMaxSlots || !g->slots[id].used) return fail(NB_ERR_ARG, "unknown request id");
    if (prec) *prec = g->h_desc[id].prec;
    if (outer) *outer = g->h_desc[id].outer;
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

nb_status nb_engine_tuning(const nb_engine *g, int n, nb_precision prec, int *lines_per_thread,
                           int *elems_per_tile) {
    if (!g || n < 2 || n > kMaxN || (prec != NB_FP64 && prec != NB_MIXED)) return fail(NB_ERR_ARG, "bad argument");
    const NGroup &G = prec == NB_MIXED ? g->mgroups[n] : g->groups[n];
    if (lines_per_thread) *lines_per_thread = G.lpt;
    if (elems_per_tile) *elems_per_tile = G.te;
    return NB_OK;
}

}  // extern "C"
